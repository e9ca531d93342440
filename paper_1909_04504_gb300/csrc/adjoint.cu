// Hand-written adjoint of the neighbour-fixed WCSPH step (reverse of the Sec. 2.1
// predictor-corrector with the density advanced like the positions):
//   forward step n -> n+1 (cell order O_n -> O_{n+1}, perm: O_{n+1} -> O_n):
//     drift  uh = u + dt/2 a, x' = x + dt (uh + xsph)          (fluid, order O_n)
//     gather x, uh, rho into O_{n+1}
//     density  rho' = rho + dt D(x, uh)                         (Eq. continuity:sph)
//     momentum (a', xsph') = M(x, uh, rho') + g                 (Eqs. mom:sph*, AV, XSPH)
//     kick   u' = uh + dt/2 a'
//   reverse (cotangents of x, u', rho', a', xsph' in O_{n+1}):
//     abar = lambda_a' + dt/2 lambda_u', lambda_uh = lambda_u'
//     momentum VJP  -> lambda_x, lambda_uh, lambda_rho' (+ Pr chain), nu-bar, alpha-bar
//     continuity VJP with cotangent dt (lambda_rho' + momentum part) -> lambda_x, lambda_uh
//     scatter to O_n and the drift transpose.
// The pair VJPs are gathers over each particle's neighbour list (the forward evaluation's,
// copied to the tape when the step is recomputed): a particle collects the
// terms where it is the destination (its own cotangents) and where it is the source (the
// neighbour's cotangents), so no atomics are needed. Pair arithmetic in the pair-loop
// precision with compensated per-particle sums; adjoint state and scalar gradients in FP64.
#include "pairs_impl.cuh"

namespace sph {

// ------------------------------------------------------------ taped lists
// Copy of the forward evaluation's neighbour list (nl[k * n + i], k < cnt[i]) into the
// tape: the reverse sweep runs over exactly the pairs the forward step summed. Only the
// filled entries move; for each k the threads of a warp touch consecutive words.
__global__ void k_tape_list(const uint32_t* __restrict__ nl, const uint32_t* __restrict__ cnt,
                            int n, uint32_t* __restrict__ tnl, uint32_t* __restrict__ tcnt) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint32_t c = cnt[i];
        tcnt[i] = c;
        for (uint32_t k = 0; k < c; ++k) tnl[(size_t)k * n + i] = nl[(size_t)k * n + i];
    }
}

// ------------------------------------------------------------- kernel derivative
// fp(q) = f'(q) / q with f = w'(q) / q the gradient factor of the pair loops, so that
// d(Gk)/dr_vec = gfac fp(q) / h^2 * r_vec.
template <class Real, int KERNEL>
__device__ __forceinline__ Real kernel_fp(Real q) {
    if (KERNEL == QUINTIC) {
        if (q < Real(1)) return Real(-150) * q + Real(240);
        const Real t3 = Real(3) - q;
        Real w1 = Real(-5) * t3 * t3 * t3 * t3;
        Real w1p = Real(20) * t3 * t3 * t3;
        if (q < Real(2)) {
            const Real t2 = Real(2) - q;
            w1 += Real(30) * t2 * t2 * t2 * t2;
            w1p -= Real(120) * t2 * t2 * t2;
        }
        return PairMath<Real>::div(w1p * q - w1, q * q * q);
    } else if (KERNEL == CUBIC_SPLINE) {
        // f = 9 q - 12 on [0,1): f' = 9; f = -3 (2-q)^2 / q on [1,2): f' = 3 (4 - q^2) / q^2
        if (q < Real(1e-6)) return Real(0);  // multiplies r_vec -> 0 (coincident particles)
        if (q < Real(1)) return PairMath<Real>::div(Real(9), q);
        return PairMath<Real>::div(Real(3) * (Real(4) - q * q), q * q * q);
    } else {
        if (q < Real(1e-6)) return Real(0);  // multiplies r_vec -> 0 (coincident particles)
        const Real t = Real(1) - Real(0.5) * q;
        return PairMath<Real>::div(Real(7.5) * t * t, q);
    }
}

// Cotangents of one destination's momentum equation: abar (acceleration), sbar (XSPH).
template <class Real>
struct MomCot {
    Real ax, ay, az, sx, sy, sz;
};

// Factors of the momentum + XSPH terms of a pair that do not depend on the cotangents and
// are the same for both orders (i, j) and (j, i): kernel values, AV, laminar and XSPH
// weights. Inputs: r2, vr = v_ij . r_ij (even in the order), densities, Pr = p / rho^2.
template <class Real>
struct PairFactors {
    Real Gk, Gp, W, rhobar, inv_rb, coef, dPi_dvr, dPi_dr2, dPi_drhobar, c0mu_rb, lam_r, Gkg2, inv_rs;
    bool av_on;
};

template <class Real, int DIM, int KERNEL>
__device__ __forceinline__ PairFactors<Real> pair_factors(Real r2, Real vr, Real rho_i, Real rho_j,
                                                          Real pr_i, Real pr_j,
                                                          const PairConst<Real>& K, int flags) {
    using M = PairMath<Real>;
    PairFactors<Real> f;
    const Real q = M::sqrt(r2) * K.inv_h;
    f.Gk = K.gfac * kernel_f<Real, KERNEL>(q);
    f.Gp = K.gfac * kernel_fp<Real, KERNEL>(q) * (K.inv_h * K.inv_h);  // dGk/dr = Gp r
    f.W = (flags & F_XSPH) ? K.wfac * kernel_w<Real, KERNEL>(q) : Real(0);
    f.rhobar = Real(0.5) * (rho_i + rho_j);
    f.inv_rb = M::rcp(f.rhobar);
    // artificial viscosity Pi = -alpha c0 mu / rhobar, mu = h vr / (r2 + 0.01 h^2), vr < 0
    Real Pi = Real(0);
    f.dPi_dvr = f.dPi_dr2 = f.dPi_drhobar = f.c0mu_rb = Real(0);
    f.av_on = (flags & F_AV) && vr < Real(0);
    if (f.av_on) {
        const Real inv_den = M::rcp(r2 + K.av_h2);
        const Real mu = K.h * vr * inv_den;
        Pi = -K.alpha_c0 * mu * f.inv_rb;
        f.dPi_dvr = -K.alpha_c0 * K.h * inv_den * f.inv_rb;
        f.dPi_dr2 = K.alpha_c0 * mu * inv_den * f.inv_rb;  // dmu/dr2 = -mu / den
        f.dPi_drhobar = -Pi * f.inv_rb;
        f.c0mu_rb = -K.c0 * mu * f.inv_rb;  // dPi/dalpha
    }
    f.coef = pr_i + pr_j + Pi;
    // laminar viscosity weight g2 = r2 / (r2 + eta h^2) and d(Gk g2)/dr = lam_r r
    f.lam_r = f.Gkg2 = Real(0);
    f.inv_rs = M::rcp(rho_i + rho_j);
    if (flags & F_LAMINAR) {
        const Real inv_den = M::rcp(r2 + K.eta_h2);
        const Real g2 = r2 * inv_den;
        const Real dg2 = K.eta_h2 * inv_den * inv_den;  // d g2 / d r2
        f.lam_r = f.Gp * g2 + f.Gk * dg2 * Real(2);
        f.Gkg2 = f.Gk * g2;
    }
    return f;
}

// VJP of the momentum + XSPH terms of the ordered pair (i dest fluid, j source) with the
// cotangents c of i, from the pair's factors. Inputs: r = x_i - x_j, v = u_i - u_j, m_j,
// whether j is fluid. Outputs (added): g_r, g_v (vectors), g_rho (the same for rho_i and
// rho_j: every density enters through rhobar or rho_i + rho_j), g_pr (the same for Pr_i
// and Pr_j); with SCALARS also g_nu and g_alpha.
template <class Real, int DIM, bool SCALARS>
__device__ __forceinline__ void momentum_vjp(Real rx, Real ry, Real rz, Real vx, Real vy, Real vz,
                                             const PairFactors<Real>& f, Real mj, bool fluid_j,
                                             const MomCot<Real>& c, const PairConst<Real>& K,
                                             int flags, Real* g_r, Real* g_v, Real& g_rho,
                                             Real& g_pr, Real& g_nu, Real& g_alpha) {
    const Real ar = c.ax * rx + c.ay * ry + (DIM == 3 ? c.az * rz : Real(0));
    // pressure + artificial viscosity: a_i += -m_j (Pr_i + Pr_j + Pi) Gk r
    // d(ar Gk coef)/dr: ar -> abar, Gk -> Gp r, coef -> dPi/dr (vr: v, r2: 2 r)
    const Real mGa = mj * f.Gk * ar;
    const Real s1 = -mj * (f.coef * f.Gp * ar + f.Gk * ar * f.dPi_dr2 * Real(2));
    const Real s2 = -mj * f.coef * f.Gk;
    const Real s3 = -mGa * f.dPi_dvr;
    g_r[0] += s1 * rx + s2 * c.ax + s3 * vx;
    g_r[1] += s1 * ry + s2 * c.ay + s3 * vy;
    if (DIM == 3) g_r[2] += s1 * rz + s2 * c.az + s3 * vz;
    g_v[0] += s3 * rx;
    g_v[1] += s3 * ry;
    if (DIM == 3) g_v[2] += s3 * rz;
    g_pr += -mGa;
    g_rho += -mGa * f.dPi_drhobar * Real(0.5);
    if (SCALARS && f.av_on) g_alpha += -mGa * f.c0mu_rb;
    // laminar viscosity: a_i += m_j 4 nu / (rho_i + rho_j) Gk g2 v
    if (flags & F_LAMINAR) {
        const Real av = c.ax * vx + c.ay * vy + (DIM == 3 ? c.az * vz : Real(0));
        const Real cvn = mj * K.nu4 * f.inv_rs;  // cv / (Gk g2)
        const Real t1 = cvn * av * f.lam_r;
        g_r[0] += t1 * rx;
        g_r[1] += t1 * ry;
        if (DIM == 3) g_r[2] += t1 * rz;
        const Real cv = cvn * f.Gkg2;
        g_v[0] += cv * c.ax;
        g_v[1] += cv * c.ay;
        if (DIM == 3) g_v[2] += cv * c.az;
        g_rho += -cv * av * f.inv_rs;
        if (SCALARS) g_nu += Real(4) * mj * f.inv_rs * f.Gkg2 * av;  // d/dnu (nu4 = 4 nu)
    }
    // XSPH over fluid sources: xs_i += -eps m_j W v / rhobar
    if ((flags & F_XSPH) && fluid_j) {
        const Real sv = c.sx * vx + c.sy * vy + (DIM == 3 ? c.sz * vz : Real(0));
        const Real e = K.xsph * mj * f.inv_rb;
        const Real t1 = -e * sv * f.Gk;  // dW/dr = Gk r
        g_r[0] += t1 * rx;
        g_r[1] += t1 * ry;
        if (DIM == 3) g_r[2] += t1 * rz;
        g_v[0] += -e * f.W * c.sx;
        g_v[1] += -e * f.W * c.sy;
        if (DIM == 3) g_v[2] += -e * f.W * c.sz;
        g_rho += e * f.W * sv * f.inv_rb * Real(0.5);
    }
}

// ------------------------------------------------------------ adjoint kernels
// Cotangent shadow of one evaluation in the taped order: CA = (abar, c_rho) and
// CS = (sbar, 0) for fluid particles (walls: zero), lambda_uh = lambda_u.
// kick = 1 adds the corrector's dt/2 lambda_u' to abar (a step); 0 for the initial
// evaluation (no kick follows it).
template <class Real>
__global__ void k_adj_cot(AdjSet L, const typename V4<Real>::T* __restrict__ P, int n, double dt,
                          int kick, typename V4<Real>::T* __restrict__ CA,
                          typename V4<Real>::T* __restrict__ CS, double* __restrict__ luh0,
                          double* __restrict__ luh1, double* __restrict__ luh2, int dim) {
    double* luh[3] = {luh0, luh1, luh2};
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        // loads first (the arrays could alias as far as the compiler knows), walls zeroed
        const bool fluid = P[k].w > Real(0);
        double la[3] = {0, 0, 0}, lu[3] = {0, 0, 0}, ls[3] = {0, 0, 0};
#pragma unroll
        for (int d = 0; d < 3; ++d)
            if (d < dim) {
                la[d] = L.a[d][k];
                lu[d] = L.u[d][k];
                ls[d] = L.xs[d][k];
            }
        typename V4<Real>::T ca, cs;
        double ab[3] = {0, 0, 0}, sb[3] = {0, 0, 0};
#pragma unroll
        for (int d = 0; d < 3; ++d)
            if (d < dim) {
                if (fluid) {
                    ab[d] = la[d] + (kick ? 0.5 * dt * lu[d] : 0.0);
                    sb[d] = ls[d];
                }
                luh[d][k] = fluid ? lu[d] : 0.0;
            }
        ca.x = (Real)ab[0]; ca.y = (Real)ab[1]; ca.z = (Real)ab[2]; ca.w = Real(0);
        cs.x = (Real)sb[0]; cs.y = (Real)sb[1]; cs.z = (Real)sb[2]; cs.w = Real(0);
        CA[k] = ca;
        CS[k] = cs;
    }
}

// Block sum of two scalars added to the running totals by the last block (fixed order).
__device__ __forceinline__ void adj_scalars(double a, double b, double* part, AdjCtl* actl) {
    __shared__ double red[PAIR_THREADS / 32][2];
    __shared__ bool last;
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        red[warp][0] = a;
        red[warp][1] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s0 = 0, s1 = 0;
        for (int w = 0; w < PAIR_THREADS / 32; ++w) {
            s0 += red[w][0];
            s1 += red[w][1];
        }
        part[2 * blockIdx.x] = s0;
        part[2 * blockIdx.x + 1] = s1;
        __threadfence();
        last = atomicAdd(&actl->ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        double s0 = 0, s1 = 0;
        const volatile double* vp = part;
        for (int bk = 0; bk < (int)gridDim.x; ++bk) {
            s0 += vp[2 * bk];
            s1 += vp[2 * bk + 1];
        }
        actl->g_nu += s0;
        actl->g_alpha += s1;
        actl->ticket = 0;
        __threadfence();
    }
}

// Momentum + XSPH VJP gather. For particle k over its list: as destination (fluid k, its
// cotangents) and as source of each fluid neighbour j (j's cotangents). Adds to
// lambda_x and lambda_uh (fluid k), writes rhom_k = d/drho' of the momentum terms (the
// Pr = p / rho^2 part through the EOS derivative), and accumulates d/dnu, d/dalpha.
template <class Real, int DIM, int KERNEL>
__global__ void __launch_bounds__(PAIR_THREADS, sizeof(Real) == 4 ? 8 : 1)
k_adj_momentum(const typename V4<Real>::T* __restrict__ P, const typename V4<Real>::T* __restrict__ Q,
               const Real* __restrict__ R, const uint32_t* __restrict__ nl,
               const uint32_t* __restrict__ cnt, int n, Grid G, PairConst<Real> K, StepConst C,
               const typename V4<Real>::T* __restrict__ CA, const typename V4<Real>::T* __restrict__ CS,
               AdjSet L, double* __restrict__ luh0, double* __restrict__ luh1,
               double* __restrict__ luh2, double* __restrict__ rhom, double* __restrict__ part,
               AdjCtl* actl) {
    double* luh[3] = {luh0, luh1, luh2};
    const int flags = K.flags;
    double s_nu = 0, s_alpha = 0;
    for (int k = blockIdx.x * PAIR_THREADS + threadIdx.x; k < n; k += gridDim.x * PAIR_THREADS) {
        const typename V4<Real>::T pk = P[k];
        const typename V4<Real>::T qk = Q[k];
        const Real prk = R[k];
        const bool fluid_k = pk.w > Real(0);
        const Real mk = fabs(pk.w);
        const typename V4<Real>::T cak = CA[k], csk = CS[k];
        const MomCot<Real> cot_k{cak.x, cak.y, cak.z, csk.x, csk.y, csk.z};
        Acc<Real> gx[3], gu[3], grho, gpr, gnu, gal;
        for (int d = 0; d < 3; ++d) {
            gx[d].zero();
            gu[d].zero();
        }
        grho.zero(); gpr.zero(); gnu.zero(); gal.zero();
        const uint32_t nk = cnt[k];
        for (uint32_t kk = 0; kk < nk; ++kk) {
            const uint32_t j = nl[(size_t)kk * n + k];
            const typename V4<Real>::T pj = P[j];
            Real rx, ry, rz;
            const Real r2 = separation<Real, DIM>(pk, pj, G, K, rx, ry, rz);
            const typename V4<Real>::T qj = Q[j];
            const Real prj = R[j];
            const bool fluid_j = pj.w > Real(0);
            const Real vx = qk.x - qj.x, vy = qk.y - qj.y, vz = DIM == 3 ? qk.z - qj.z : Real(0);
            const Real vr = vx * rx + vy * ry + (DIM == 3 ? vz * rz : Real(0));
            // the factors of the pair serve both orders: (k, j) and (j, k)
            const PairFactors<Real> f =
                pair_factors<Real, DIM, KERNEL>(r2, vr, qk.w, qj.w, prk, prj, K, flags);
            // both roles summed before the compensated accumulation
            Real g_r[3] = {0, 0, 0}, g_v[3] = {0, 0, 0}, g_rho = 0, g_p = 0, g_n = 0, g_a = 0;
            if (fluid_k)  // k is the destination
                momentum_vjp<Real, DIM, true>(rx, ry, rz, vx, vy, vz, f, fabs(pj.w), fluid_j,
                                              cot_k, K, flags, g_r, g_v, g_rho, g_p, g_n, g_a);
            if (fluid_j) {  // k is the source of destination j: d/dx_k = -d/dr
                const typename V4<Real>::T caj = CA[j], csj = CS[j];
                const MomCot<Real> cot_j{caj.x, caj.y, caj.z, csj.x, csj.y, csj.z};
                Real h_r[3] = {0, 0, 0}, h_v[3] = {0, 0, 0};
                momentum_vjp<Real, DIM, false>(-rx, -ry, -rz, -vx, -vy, -vz, f, mk, fluid_k, cot_j,
                                               K, flags, h_r, h_v, g_rho, g_p, g_n, g_a);
                for (int d = 0; d < DIM; ++d) {
                    g_r[d] -= h_r[d];
                    g_v[d] -= h_v[d];
                }
            }
            for (int d = 0; d < DIM; ++d) {
                gx[d].add(g_r[d]);
                gu[d].add(g_v[d]);
            }
            grho.add(g_rho);
            gpr.add(g_p);
            if (fluid_k) {
                gnu.add(g_n);
                gal.add(g_a);
            }
        }
        if (fluid_k) {  // read-modify-write: every read before the first write
            double lx[DIM], lu[DIM];
#pragma unroll
            for (int d = 0; d < DIM; ++d) {
                lx[d] = L.x[d][k];
                lu[d] = luh[d][k];
            }
#pragma unroll
            for (int d = 0; d < DIM; ++d) {
                L.x[d][k] = lx[d] + gx[d].value();
                luh[d][k] = lu[d] + gu[d].value();
            }
        }
        // EOS chain: d(p / rho^2)/drho = c0^2 (rho/rho0)^(gamma-1) / rho^2 - 2 p / rho^3
        const double rho = (double)qk.w;
        const double p = tait_pressure(rho, C);
        const double x = rho * C.inv_rho0;
        double xg1;  // (rho / rho0)^(gamma - 1)
        if (C.gamma7) {
            const double x3 = x * x * x;
            xg1 = x3 * x3;
        } else {
            xg1 = pow(x, C.gamma - 1.0);
        }
        const double dp = C.c0 * C.c0 * xg1;
        const double dpr = dp / (rho * rho) - 2.0 * p / (rho * rho * rho);
        rhom[k] = grho.value() + dpr * gpr.value();
        s_nu += gnu.value();
        s_alpha += gal.value();
    }
    adj_scalars(s_nu, s_alpha, part, actl);
}

// Continuity cotangent c_k = dt lambda_rho'_total,k and the total density adjoint.
template <class Real>
__global__ void k_adj_rho(AdjSet L, const double* __restrict__ rhom, int n, double dt,
                          typename V4<Real>::T* __restrict__ CA, double* __restrict__ lrho_tot) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const double t = L.rho[k] + rhom[k];
        lrho_tot[k] = t;
        reinterpret_cast<Real*>(&CA[k])[3] = (Real)(dt * t);
    }
}

// Continuity VJP gather: arho_i = sum_j m_j Gk_ij (v_ij . r_ij) over interacting pairs.
// Both roles of k combine into (c_k m_j + c_j m_k) (Gp vr r + Gk v) for lambda_x and
// (c_k m_j + c_j m_k) Gk r for lambda_uh (fluid k).
template <class Real, int DIM, int KERNEL>
__global__ void __launch_bounds__(PAIR_THREADS)
k_adj_continuity(const typename V4<Real>::T* __restrict__ P, const typename V4<Real>::T* __restrict__ Q,
                 const uint32_t* __restrict__ nl, const uint32_t* __restrict__ cnt, int n, Grid G,
                 PairConst<Real> K, const typename V4<Real>::T* __restrict__ CA, AdjSet L,
                 double* __restrict__ luh0, double* __restrict__ luh1, double* __restrict__ luh2) {
    double* luh[3] = {luh0, luh1, luh2};
    for (int k = blockIdx.x * PAIR_THREADS + threadIdx.x; k < n; k += gridDim.x * PAIR_THREADS) {
        const typename V4<Real>::T pk = P[k];
        if (!(pk.w > Real(0))) continue;  // walls: x and u are constants
        const typename V4<Real>::T qk = Q[k];
        const Real mk = fabs(pk.w);
        const Real ck = reinterpret_cast<const Real*>(&CA[k])[3];
        Acc<Real> gx[3], gu[3];
        for (int d = 0; d < 3; ++d) {
            gx[d].zero();
            gu[d].zero();
        }
        const uint32_t nk = cnt[k];
        for (uint32_t kk = 0; kk < nk; ++kk) {
            const uint32_t j = nl[(size_t)kk * n + k];
            const typename V4<Real>::T pj = P[j];
            Real rx, ry, rz;
            const Real r2 = separation<Real, DIM>(pk, pj, G, K, rx, ry, rz);
            const typename V4<Real>::T qj = Q[j];
            const Real cj = reinterpret_cast<const Real*>(&CA[j])[3];
            const Real q = PairMath<Real>::sqrt(r2) * K.inv_h;
            const Real Gk = K.gfac * kernel_f<Real, KERNEL>(q);
            const Real Gp = K.gfac * kernel_fp<Real, KERNEL>(q) * (K.inv_h * K.inv_h);
            const Real vx = qk.x - qj.x, vy = qk.y - qj.y, vz = DIM == 3 ? qk.z - qj.z : Real(0);
            const Real vr = vx * rx + vy * ry + (DIM == 3 ? vz * rz : Real(0));
            const Real w = ck * fabs(pj.w) + cj * mk;
            const Real a = w * Gp * vr, b = w * Gk;
            gx[0].add(a * rx + b * vx);
            gx[1].add(a * ry + b * vy);
            if (DIM == 3) gx[2].add(a * rz + b * vz);
            gu[0].add(b * rx);
            gu[1].add(b * ry);
            if (DIM == 3) gu[2].add(b * rz);
        }
        double lx[DIM], lu[DIM];  // read-modify-write: every read before the first write
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            lx[d] = L.x[d][k];
            lu[d] = luh[d][k];
        }
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            L.x[d][k] = lx[d] + gx[d].value();
            luh[d][k] = lu[d] + gu[d].value();
        }
    }
}

// Transpose of the gather (O_n <- O_{n+1}) and of the drift/kick of the previous state:
// uh = u + dt/2 a feeds both the evaluation (lambda_uh) and x' = x + dt (uh + xsph).
__global__ void k_adj_scatter(AdjSet in, AdjSet out, const double* __restrict__ luh0,
                              const double* __restrict__ luh1, const double* __restrict__ luh2,
                              const double* __restrict__ lrho_tot, const uint32_t* __restrict__ perm,
                              const uint32_t* __restrict__ tag, int n, int dim, double dt) {
    const double* luh[3] = {luh0, luh1, luh2};
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        // loads first (the arrays could alias as far as the compiler knows), walls zeroed
        const int o = (int)perm[k];
        const bool fluid = !(tag[k] & WALL_BIT);
        double lx[3] = {0, 0, 0}, lu[3] = {0, 0, 0};
#pragma unroll
        for (int d = 0; d < 3; ++d)
            if (d < dim) {
                lx[d] = in.x[d][k];
                lu[d] = luh[d][k];
            }
        const double lr = lrho_tot[k];
#pragma unroll
        for (int d = 0; d < 3; ++d)
            if (d < dim) {
                const double x = fluid ? lx[d] : 0.0, u = fluid ? lu[d] : 0.0;
                out.x[d][o] = x;
                out.u[d][o] = u + dt * x;
                out.a[d][o] = 0.5 * dt * u + 0.5 * dt * dt * x;
                out.xs[d][o] = dt * x;
            }
        out.rho[o] = lr;
    }
}

// Final adjoint of the initial velocities, scattered to global ids: out[d * n + id].
__global__ void k_adj_to_original(const double* __restrict__ luh0, const double* __restrict__ luh1,
                                  const double* __restrict__ luh2, const uint32_t* __restrict__ tag,
                                  int n, int dim, double* __restrict__ out) {
    const double* luh[3] = {luh0, luh1, luh2};
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const uint32_t t = tag[k];
        const uint32_t id = t & ID_MASK;
        const bool fluid = !(t & WALL_BIT);
        for (int d = 0; d < dim; ++d) out[(size_t)d * n + id] = fluid ? luh[d][k] : 0.0;
    }
}

// Terminal cotangent of KE = 1/2 sum_fluid m |u|^2 in the final order: lambda_u = m u.
__global__ void k_adj_terminal(AdjSet L, ParticleSet S, int n, int dim) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const bool fluid = !(S.tag[k] & WALL_BIT);
        for (int d = 0; d < 3; ++d) {
            L.x[d][k] = 0.0;
            L.u[d][k] = (fluid && d < dim) ? S.m[k] * S.u[d][k] : 0.0;
            L.a[d][k] = 0.0;
            L.xs[d][k] = 0.0;
        }
        L.rho[k] = 0.0;
    }
}

// ---------------------------------------------------------------- launchers
static inline int grid_of(long long n, int threads, int cap) {
    long long b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    return (int)(b > cap ? cap : b);
}

template <class Real, int DIM, int KERNEL>
static void adj_eval_t(const AdjLaunch& A, const PairConst<Real>& K, cudaStream_t st) {
    using V = typename V4<Real>::T;
    const int g256 = grid_of(A.n, 256, A.sms * 8);
    const int gp = grid_of(A.n, PAIR_THREADS, A.sms * 16);
    k_adj_cot<Real><<<g256, 256, 0, st>>>(A.L, (const V*)A.P, A.n, A.dt, A.kick, (V*)A.CA,
                                          (V*)A.CS, A.luh[0], A.luh[1], A.luh[2], DIM);
    k_adj_momentum<Real, DIM, KERNEL><<<gp, PAIR_THREADS, 0, st>>>(
        (const V*)A.P, (const V*)A.Q, (const Real*)A.R, A.nl, A.cnt, A.n, A.G, K, A.C,
        (const V*)A.CA, (const V*)A.CS, A.L, A.luh[0], A.luh[1], A.luh[2], A.rhom, A.part, A.actl);
    k_adj_rho<Real><<<g256, 256, 0, st>>>(A.L, A.rhom, A.n, A.kick ? A.dt : 0.0, (V*)A.CA,
                                          A.lrho_tot);
    if (A.kick)
        k_adj_continuity<Real, DIM, KERNEL><<<gp, PAIR_THREADS, 0, st>>>(
            (const V*)A.P, (const V*)A.Q, A.nl, A.cnt, A.n, A.G, K, (const V*)A.CA, A.L, A.luh[0],
            A.luh[1], A.luh[2]);
}

void launch_adjoint_eval(const AdjLaunch& A, const PairConst<float>& Kf, const PairConst<double>& Kd,
                         cudaStream_t st) {
    const int sel = (A.precision ? 6 : 0) + (A.dim == 3 ? 3 : 0) + A.kernel;
    switch (sel) {
        case 0: adj_eval_t<double, 2, QUINTIC>(A, Kd, st); break;
        case 1: adj_eval_t<double, 2, WENDLAND_C2>(A, Kd, st); break;
        case 2: adj_eval_t<double, 2, CUBIC_SPLINE>(A, Kd, st); break;
        case 3: adj_eval_t<double, 3, QUINTIC>(A, Kd, st); break;
        case 4: adj_eval_t<double, 3, WENDLAND_C2>(A, Kd, st); break;
        case 5: adj_eval_t<double, 3, CUBIC_SPLINE>(A, Kd, st); break;
        case 6: adj_eval_t<float, 2, QUINTIC>(A, Kf, st); break;
        case 7: adj_eval_t<float, 2, WENDLAND_C2>(A, Kf, st); break;
        case 8: adj_eval_t<float, 2, CUBIC_SPLINE>(A, Kf, st); break;
        case 9: adj_eval_t<float, 3, QUINTIC>(A, Kf, st); break;
        case 10: adj_eval_t<float, 3, WENDLAND_C2>(A, Kf, st); break;
        default: adj_eval_t<float, 3, CUBIC_SPLINE>(A, Kf, st); break;
    }
}

void launch_tape_list(const uint32_t* nl, const uint32_t* cnt, int n, uint32_t* tnl, uint32_t* tcnt,
                      int sms, cudaStream_t st) {
    k_tape_list<<<grid_of(n, 256, sms * 8), 256, 0, st>>>(nl, cnt, n, tnl, tcnt);
}

void launch_adjoint_scatter(const AdjLaunch& A, const AdjSet& out, cudaStream_t st) {
    k_adj_scatter<<<grid_of(A.n, 256, A.sms * 8), 256, 0, st>>>(
        A.L, out, A.luh[0], A.luh[1], A.luh[2], A.lrho_tot, A.perm, A.tag, A.n, A.dim, A.dt);
}

void launch_adjoint_terminal(const AdjSet& L, const ParticleSet& S, int n, int dim, int sms,
                             cudaStream_t st) {
    k_adj_terminal<<<grid_of(n, 256, sms * 8), 256, 0, st>>>(L, S, n, dim);
}

void launch_adjoint_to_original(const AdjLaunch& A, double* out, cudaStream_t st) {
    k_adj_to_original<<<grid_of(A.n, 256, A.sms * 8), 256, 0, st>>>(A.luh[0], A.luh[1], A.luh[2],
                                                                     A.tag, A.n, A.dim, out);
}

int adjoint_partial_blocks(int n, int sms) { return grid_of(n, PAIR_THREADS, sms * 16); }

}  // namespace sph
