// Pair loops of one right-hand-side evaluation over the cell-sorted particles
// (Sec. 3.2 groups; pseudo-code of the per-destination loop in Sec. 3.4):
//  - summation density, Eq. (2), followed by the EOS, Eq. (eos);
//  - the fused loop: continuity Eq. (continuity:sph), pressure Eq. (mom:sph:press),
//    laminar viscosity Eq. (mom:sph:visc), Monaghan artificial viscosity, XSPH, plus
//    the body force of Eq. (mom:sph), with the corrector half-kick of Sec. 2.1 and the
//    FP64 diagnostics reduction fused into the epilogue.
// One thread owns one destination particle and walks the 3^(d-1) contiguous source
// runs of its stencil (a row of three cells is contiguous in the sorted order).
#include "sph_device.cuh"
#include "sph_launch.h"

namespace sph {

constexpr int PAIR_THREADS = 128;
constexpr int PARTIAL_STRIDE = 16;  // doubles per block partial

// Walks the stencil of cell (cx, cy, cz): calls body(jb, je) for each contiguous run.
template <int DIM, class Body>
__device__ __forceinline__ void for_each_run(const Grid& G, const uint32_t* __restrict__ off,
                                             int cx, int cy, int cz, Body body) {
#pragma unroll 1
    for (int dz = (DIM == 3 ? -1 : 0); dz <= (DIM == 3 ? 1 : 0); ++dz) {
        int z = cz + dz;
        if (DIM == 3 && (z < 0 || z >= G.nc[2])) {
            if (!G.periodic[2]) continue;
            z = (z + G.nc[2]) % G.nc[2];
        }
#pragma unroll 1
        for (int dy = -1; dy <= 1; ++dy) {
            int y = cy + dy;
            if (y < 0 || y >= G.nc[1]) {
                if (!G.periodic[1]) continue;
                y = (y + G.nc[1]) % G.nc[1];
            }
            const int row = G.nc[0] * (y + G.nc[1] * z);
            int x0 = cx - 1, x1 = cx + 1;
            if (G.periodic[0]) {
                if (x0 < 0) { body(off[row + G.nc[0] - 1], off[row + G.nc[0]]); x0 = 0; }
                if (x1 >= G.nc[0]) { body(off[row], off[row + 1]); x1 = G.nc[0] - 1; }
            } else {
                if (x0 < 0) x0 = 0;
                if (x1 >= G.nc[0]) x1 = G.nc[0] - 1;
            }
            body(off[row + x0], off[row + x1 + 1]);
        }
    }
}

__device__ __forceinline__ void cell_of_key(const Grid& G, uint32_t key, int& cx, int& cy, int& cz) {
    cx = (int)(key % (uint32_t)G.nc[0]);
    uint32_t r = key / (uint32_t)G.nc[0];
    cy = (int)(r % (uint32_t)G.nc[1]);
    cz = (int)(r / (uint32_t)G.nc[1]);
}

// ------------------------------------------------------ summation density
template <class Real, int DIM, int KERNEL>
__global__ void __launch_bounds__(PAIR_THREADS)
k_density(const typename V4<Real>::T* __restrict__ P, typename V4<Real>::T* __restrict__ Q,
          Real* __restrict__ R, const uint32_t* __restrict__ skeys, const uint32_t* __restrict__ off,
          int n, Grid G, PairConst<Real> K, StepConst C, ParticleSet S, const Control* ctl) {
    if (ctl->status) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const typename V4<Real>::T pi = P[i];
        int cx, cy, cz;
        cell_of_key(G, skeys[i], cx, cy, cz);
        Acc<Real> sum;
        sum.zero();
        sum.add(fabs(pi.w) * K.wfac * kernel_w<Real, KERNEL>(Real(0)));
        for_each_run<DIM>(G, off, cx, cy, cz, [&](uint32_t jb, uint32_t je) {
            for (uint32_t j = jb; j < je; ++j) {
                if ((int)j == i) continue;
                const typename V4<Real>::T pj = P[j];
                Real dx = min_image(rn_sub(pi.x, pj.x), G.periodic[0], K.L[0], K.halfL[0]);
                Real dy = min_image(rn_sub(pi.y, pj.y), G.periodic[1], K.L[1], K.halfL[1]);
                Real dz = DIM == 3 ? min_image(rn_sub(pi.z, pj.z), G.periodic[2], K.L[2], K.halfL[2]) : Real(0);
                Real r2 = dist2<Real, DIM>(dx, dy, dz);
                if (!(r2 < K.kh2)) continue;
                Real q = sqrt(r2) * K.inv_h;
                sum.add(fabs(pj.w) * K.wfac * kernel_w<Real, KERNEL>(q));
            }
        });
        const double rho = sum.value();
        S.rho[i] = rho;
        double r = rho * C.inv_rho0;
        double rg;
        if (C.gamma7) {
            double r2 = r * r;
            rg = r2 * r2 * r2 * r;
        } else {
            rg = pow(r, C.gamma);
        }
        const double p = C.B * (rg - 1.0);
        typename V4<Real>::T qi = Q[i];
        qi.w = (Real)rho;
        Q[i] = qi;
        R[i] = (Real)(p / (rho * rho));
    }
}

// ------------------------------------------------------------ fused pair loop
template <class Real, int DIM, int KERNEL>
__global__ void __launch_bounds__(PAIR_THREADS)
k_pairs(const typename V4<Real>::T* __restrict__ P, const typename V4<Real>::T* __restrict__ Q,
        const Real* __restrict__ R, const uint32_t* __restrict__ skeys,
        const uint32_t* __restrict__ off, int n, Grid G, PairConst<Real> K, StepConst C,
        ParticleSet S, Control* ctl, int kick, double* __restrict__ partials,
        double* __restrict__ history) {
    if (ctl->status) return;
    const double dt = ctl->dt;
    const int flags = K.flags;
    double d_px = 0, d_py = 0, d_pz = 0, d_ke = 0, d_u2 = 0, d_a2 = 0, d_pairs = 0, d_cand = 0;
    int bad = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const typename V4<Real>::T pi = P[i];
        const typename V4<Real>::T qi = Q[i];
        const Real pri = R[i];
        const bool fluid_i = pi.w > Real(0);
        int cx, cy, cz;
        cell_of_key(G, skeys[i], cx, cy, cz);
        Acc<Real> arho, ax, ay, az, sx, sy, sz;
        arho.zero(); ax.zero(); ay.zero(); az.zero(); sx.zero(); sy.zero(); sz.zero();
        uint32_t npairs = 0, ncand = 0;
        for_each_run<DIM>(G, off, cx, cy, cz, [&](uint32_t jb, uint32_t je) {
            for (uint32_t j = jb; j < je; ++j) {
                if ((int)j == i) continue;
                ++ncand;
                const typename V4<Real>::T pj = P[j];
                Real dx = min_image(rn_sub(pi.x, pj.x), G.periodic[0], K.L[0], K.halfL[0]);
                Real dy = min_image(rn_sub(pi.y, pj.y), G.periodic[1], K.L[1], K.halfL[1]);
                Real dz = DIM == 3 ? min_image(rn_sub(pi.z, pj.z), G.periodic[2], K.L[2], K.halfL[2]) : Real(0);
                Real r2 = dist2<Real, DIM>(dx, dy, dz);
                if (!(r2 < K.kh2)) continue;
                const bool fluid_j = pj.w > Real(0);
                if (!fluid_i && !fluid_j) continue;  // wall-wall pairs carry no equation
                ++npairs;
                const typename V4<Real>::T qj = Q[j];
                const Real mj = fabs(pj.w);
                const Real q = sqrt(r2) * K.inv_h;
                const Real Gk = K.gfac * kernel_f<Real, KERNEL>(q);  // grad_i W = Gk (x_i - x_j)
                const Real vx = qi.x - qj.x, vy = qi.y - qj.y, vz = DIM == 3 ? qi.z - qj.z : Real(0);
                const Real vdotr = vx * dx + vy * dy + (DIM == 3 ? vz * dz : Real(0));
                if (flags & F_CONTINUITY) arho.add(mj * Gk * vdotr);
                if (!fluid_i) continue;
                Real coef = pri + R[j];
                const Real rhobar = Real(0.5) * (qi.w + qj.w);
                if ((flags & F_AV) && vdotr < Real(0)) {
                    const Real mu = K.h * vdotr / (r2 + K.av_h2);
                    coef -= K.alpha_c0 * mu / rhobar;
                }
                const Real cg = -mj * coef * Gk;
                Real cv = Real(0);
                if (flags & F_LAMINAR) cv = mj * K.nu4 / (qi.w + qj.w) * Gk * r2 / (r2 + K.eta_h2);
                ax.add(cg * dx + cv * vx);
                ay.add(cg * dy + cv * vy);
                if (DIM == 3) az.add(cg * dz + cv * vz);
                if ((flags & F_XSPH) && fluid_j) {
                    const Real fx = K.xsph * mj / rhobar * (K.wfac * kernel_w<Real, KERNEL>(q));
                    sx.add(-fx * vx);
                    sy.add(-fx * vy);
                    if (DIM == 3) sz.add(-fx * vz);
                }
            }
        });
        // epilogue: FP64 rates, corrector half-kick, diagnostics
        double a[3] = {ax.value(), ay.value(), az.value()};
        double xs[3] = {sx.value(), sy.value(), sz.value()};
        const double ar = arho.value();
        if (fluid_i)
            for (int d = 0; d < DIM; ++d) a[d] += C.g[d];
        S.arho[i] = ar;
        for (int d = 0; d < DIM; ++d) {
            S.a[d][i] = a[d];
            S.xs[d][i] = xs[d];
        }
        double u[3] = {0, 0, 0};
        for (int d = 0; d < DIM; ++d) {
            u[d] = S.u[d][i];
            if (kick && fluid_i) {
                u[d] += 0.5 * dt * a[d];
                S.u[d][i] = u[d];
            }
        }
        double rho = S.rho[i];
        if (kick && C.continuity) {
            rho += 0.5 * dt * ar;
            S.rho[i] = rho;
        }
        if (!isfinite(rho) || !isfinite(ar)) bad = 1;
        if (fluid_i) {
            const double m = S.m[i];
            double u2 = 0, a2 = 0;
            for (int d = 0; d < DIM; ++d) {
                u2 += u[d] * u[d];
                a2 += a[d] * a[d];
                if (!isfinite(u[d]) || !isfinite(S.x[d][i])) bad = 1;
            }
            d_px += m * u[0];
            d_py += m * u[1];
            d_pz += m * u[2];
            d_ke += 0.5 * m * u2;
            d_u2 = fmax(d_u2, u2);
            d_a2 = fmax(d_a2, a2);
            if (!isfinite(a2)) bad = 1;
        }
        d_pairs += (double)npairs;
        d_cand += (double)ncand;
    }

    // ---- block reduction (fixed tree order: deterministic)
    __shared__ double red[PAIR_THREADS / 32][10];
    __shared__ bool is_last;
    double v[10] = {d_px, d_py, d_pz, d_ke, d_u2, d_a2, d_pairs, d_cand, (double)bad, 0.0};
    for (int o = 16; o > 0; o >>= 1) {
        for (int k = 0; k < 9; ++k) {
            double y = __shfl_down_sync(0xffffffffu, v[k], o);
            v[k] = (k == 4 || k == 5 || k == 8) ? fmax(v[k], y) : v[k] + y;
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0)
        for (int k = 0; k < 9; ++k) red[warp][k] = v[k];
    __syncthreads();
    if (threadIdx.x == 0) {
        double out[9];
        for (int k = 0; k < 9; ++k) out[k] = red[0][k];
        for (int w = 1; w < PAIR_THREADS / 32; ++w)
            for (int k = 0; k < 9; ++k)
                out[k] = (k == 4 || k == 5 || k == 8) ? fmax(out[k], red[w][k]) : out[k] + red[w][k];
        for (int k = 0; k < 9; ++k) partials[(size_t)blockIdx.x * PARTIAL_STRIDE + k] = out[k];
        __threadfence();
        unsigned t = atomicAdd(&ctl->ticket, 1u);
        is_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    // ---- last block: reduce the partials in a fixed order and finalise
    for (int k = 0; k < 9; ++k) v[k] = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
        const volatile double* p = partials + (size_t)b * PARTIAL_STRIDE;
        for (int k = 0; k < 9; ++k) {
            double y = p[k];
            v[k] = (k == 4 || k == 5 || k == 8) ? fmax(v[k], y) : v[k] + y;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        for (int k = 0; k < 9; ++k) {
            double y = __shfl_down_sync(0xffffffffu, v[k], o);
            v[k] = (k == 4 || k == 5 || k == 8) ? fmax(v[k], y) : v[k] + y;
        }
    }
    __syncthreads();
    if (lane == 0)
        for (int k = 0; k < 9; ++k) red[warp][k] = v[k];
    __syncthreads();
    if (threadIdx.x == 0) {
        double out[9];
        for (int k = 0; k < 9; ++k) out[k] = red[0][k];
        for (int w = 1; w < PAIR_THREADS / 32; ++w)
            for (int k = 0; k < 9; ++k)
                out[k] = (k == 4 || k == 5 || k == 8) ? fmax(out[k], red[w][k]) : out[k] + red[w][k];
        ctl->ticket = 0;
        double* rec = ctl->rec;
        if (kick) {
            ctl->t += dt;
            ctl->step += 1;
        }
        rec[0] = ctl->t;
        rec[1] = kick ? dt : 0.0;
        rec[2] = out[3];
        rec[3] = sqrt(out[4]);
        rec[4] = out[0];
        rec[5] = out[1];
        rec[6] = out[2];
        rec[7] = sqrt(out[5]);
        rec[8] = out[6];
        rec[9] = out[7];
        rec[10] = (double)ctl->step;
        rec[11] = (double)ctl->outside;
        if (out[8] != 0.0) ctl->status |= ST_NONFINITE;
        double dt_next = C.dt_fixed;
        if (!(dt_next > 0.0)) {
            dt_next = 0.25 * C.h / (C.c0 + rec[3]);
            if (rec[7] > 0.0) dt_next = fmin(dt_next, 0.25 * sqrt(C.h / rec[7]));
            if (C.nu > 0.0) dt_next = fmin(dt_next, 0.125 * C.h * C.h / C.nu);
        }
        ctl->dt = dt_next;
        if (kick) {
            double* hrec = history + (size_t)(ctl->hist_count % HIST_CAP) * DIAG_N;
            for (int k = 0; k < DIAG_N; ++k) hrec[k] = rec[k];
            ctl->hist_count += 1;
        }
        __threadfence();
    }
}

// ---------------------------------------------------------------- launchers
template <class Real, int DIM, int KERNEL>
static void pairs_t(const PairLaunch& L, const PairConst<Real>& K, cudaStream_t st) {
    using V = typename V4<Real>::T;
    if (L.summation)
        k_density<Real, DIM, KERNEL><<<L.grid, PAIR_THREADS, 0, st>>>(
            (const V*)L.P, (V*)L.Q, (Real*)L.R, L.skeys, L.off, L.n, L.G, K, L.C, L.S, L.ctl);
    k_pairs<Real, DIM, KERNEL><<<L.grid, PAIR_THREADS, 0, st>>>(
        (const V*)L.P, (const V*)L.Q, (const Real*)L.R, L.skeys, L.off, L.n, L.G, K, L.C, L.S,
        L.ctl, L.kick, L.partials, L.history);
}

int pair_threads() { return PAIR_THREADS; }
int partial_stride() { return PARTIAL_STRIDE; }

void launch_pairs(const PairLaunch& L, const PairConst<float>& Kf, const PairConst<double>& Kd,
                  cudaStream_t st) {
    const int sel = (L.precision ? 4 : 0) + (L.dim == 3 ? 2 : 0) + (L.kernel == WENDLAND_C2 ? 1 : 0);
    switch (sel) {
        case 0: pairs_t<double, 2, QUINTIC>(L, Kd, st); break;
        case 1: pairs_t<double, 2, WENDLAND_C2>(L, Kd, st); break;
        case 2: pairs_t<double, 3, QUINTIC>(L, Kd, st); break;
        case 3: pairs_t<double, 3, WENDLAND_C2>(L, Kd, st); break;
        case 4: pairs_t<float, 2, QUINTIC>(L, Kf, st); break;
        case 5: pairs_t<float, 2, WENDLAND_C2>(L, Kf, st); break;
        case 6: pairs_t<float, 3, QUINTIC>(L, Kf, st); break;
        default: pairs_t<float, 3, WENDLAND_C2>(L, Kf, st); break;
    }
}

int pairs_max_blocks_per_sm(int precision, int dim, int kernel) {
    int b = 0;
    const int sel = (precision ? 4 : 0) + (dim == 3 ? 2 : 0) + (kernel == WENDLAND_C2 ? 1 : 0);
    switch (sel) {
        case 0: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_pairs<double, 2, QUINTIC>, PAIR_THREADS, 0); break;
        case 1: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_pairs<double, 2, WENDLAND_C2>, PAIR_THREADS, 0); break;
        case 2: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_pairs<double, 3, QUINTIC>, PAIR_THREADS, 0); break;
        case 3: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_pairs<double, 3, WENDLAND_C2>, PAIR_THREADS, 0); break;
        case 4: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_pairs<float, 2, QUINTIC>, PAIR_THREADS, 0); break;
        case 5: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_pairs<float, 2, WENDLAND_C2>, PAIR_THREADS, 0); break;
        case 6: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_pairs<float, 3, QUINTIC>, PAIR_THREADS, 0); break;
        default: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_pairs<float, 3, WENDLAND_C2>, PAIR_THREADS, 0); break;
    }
    return b > 0 ? b : 1;
}

}  // namespace sph
