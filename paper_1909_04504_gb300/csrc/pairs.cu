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

// Block sum of up to 3 counters into partials[blockIdx.x * PARTIAL_STRIDE + first + k]
// (fixed tree order).
__device__ __forceinline__ void block_counts(double c0, double c1, double c2, double* partials,
                                             int first) {
    __shared__ double red[PAIR_THREADS / 32][3];
    double v[3] = {c0, c1, c2};
    for (int o = 16; o > 0; o >>= 1)
        for (int k = 0; k < 3; ++k) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0)
        for (int k = 0; k < 3; ++k) red[warp][k] = v[k];
    __syncthreads();
    if (threadIdx.x == 0)
        for (int k = 0; k < 3; ++k) {
            double t = red[0][k];
            for (int w = 1; w < PAIR_THREADS / 32; ++w) t += red[w][k];
            partials[(size_t)blockIdx.x * PARTIAL_STRIDE + first + k] = t;
        }
}

// ---------------------------------------------------------------- density pass
// First group of an evaluation (Sec. 3.2): the density of every particle, then the EOS.
//  summation (Eq. 2): rho_i = sum_j m_j W_ij, self term included;
//  continuity (Eq. continuity:sph): arho_i = sum_j m_j v_ij . grad_i W_ij (walls take
//    fluid sources only) and, inside a step, rho_i += dt arho_i, advancing the density
//    like the positions with the half-step velocities (Sec. 2.1 reading).
// Then p = B ((rho/rho0)^gamma - 1) in FP64 and the shadow rho, p / rho^2. Counts the
// interacting pairs (i != j inside the support, not both walls) and the candidates.
template <class Real, int DIM, int KERNEL>
__global__ void __launch_bounds__(PAIR_THREADS)
k_density(const typename V4<Real>::T* __restrict__ P, typename V4<Real>::T* __restrict__ Q,
          Real* __restrict__ R, const uint32_t* __restrict__ skeys, const uint32_t* __restrict__ off,
          int n, Grid G, PairConst<Real> K, StepConst C, ParticleSet S, const Control* ctl,
          int kick, double* __restrict__ partials) {
    if (ctl->status) return;
    const double dt = ctl->dt;
    const bool summation = !(K.flags & F_CONTINUITY);
    double c_pairs = 0, c_cand = 0, c_wall = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const typename V4<Real>::T pi = P[i];
        const typename V4<Real>::T qi = Q[i];
        const bool fluid_i = pi.w > Real(0);
        int cx, cy, cz;
        cell_of_key(G, skeys[i], cx, cy, cz);
        Acc<Real> sum;
        sum.zero();
        if (summation) sum.add(fabs(pi.w) * K.wfac * kernel_w<Real, KERNEL>(Real(0)));
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
                const bool interacting = fluid_i || pj.w > Real(0);
                npairs += interacting;
                const Real q = sqrt(r2) * K.inv_h;
                if (summation) {
                    sum.add(fabs(pj.w) * K.wfac * kernel_w<Real, KERNEL>(q));
                } else if (interacting) {
                    const typename V4<Real>::T qj = Q[j];
                    const Real Gk = K.gfac * kernel_f<Real, KERNEL>(q);
                    const Real vdotr = (qi.x - qj.x) * dx + (qi.y - qj.y) * dy +
                                       (DIM == 3 ? (qi.z - qj.z) * dz : Real(0));
                    sum.add(fabs(pj.w) * Gk * vdotr);
                }
            }
        });
        double rho;
        if (summation) {
            rho = sum.value();
            S.arho[i] = 0.0;
        } else {
            const double ar = sum.value();
            S.arho[i] = ar;
            rho = S.rho[i];
            if (kick) rho += dt * ar;
        }
        S.rho[i] = rho;
        const double p = tait_pressure(rho, C);
        reinterpret_cast<Real*>(&Q[i])[3] = (Real)rho;
        R[i] = (Real)(p / (rho * rho));
        c_pairs += (double)npairs;
        c_cand += (double)ncand;
        if (!fluid_i) c_wall += (double)npairs;
    }
    block_counts(c_pairs, c_cand, c_wall, partials, 10);
}

// ------------------------------------------------------------ momentum pass
// Second group of an evaluation: for every fluid destination, pressure Eq.
// (mom:sph:press), laminar viscosity Eq. (mom:sph:visc), Monaghan artificial viscosity,
// XSPH over fluid sources, the body force of Eq. (mom:sph); then, inside a step, the
// corrector half-kick u^{n+1} = u^{n+1/2} + dt/2 a^{n+1} (Sec. 2.1) and the FP64
// diagnostics. The last block to finish reduces the block partials in a fixed order
// (deterministic), writes the record, the next dt and the non-finite status.
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
    double d_px = 0, d_py = 0, d_pz = 0, d_ke = 0, d_u2 = 0, d_a2 = 0;
    int bad = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const typename V4<Real>::T pi = P[i];
        const bool fluid_i = pi.w > Real(0);
        if (!fluid_i) {  // walls: no momentum equation, static
            for (int d = 0; d < DIM; ++d) {
                S.a[d][i] = 0.0;
                S.xs[d][i] = 0.0;
            }
            if (!isfinite(S.rho[i])) bad = 1;
            continue;
        }
        const typename V4<Real>::T qi = Q[i];
        const Real pri = R[i];
        int cx, cy, cz;
        cell_of_key(G, skeys[i], cx, cy, cz);
        Acc<Real> ax, ay, az, sx, sy, sz;
        ax.zero(); ay.zero(); az.zero(); sx.zero(); sy.zero(); sz.zero();
        for_each_run<DIM>(G, off, cx, cy, cz, [&](uint32_t jb, uint32_t je) {
            for (uint32_t j = jb; j < je; ++j) {
                if ((int)j == i) continue;
                const typename V4<Real>::T pj = P[j];
                Real dx = min_image(rn_sub(pi.x, pj.x), G.periodic[0], K.L[0], K.halfL[0]);
                Real dy = min_image(rn_sub(pi.y, pj.y), G.periodic[1], K.L[1], K.halfL[1]);
                Real dz = DIM == 3 ? min_image(rn_sub(pi.z, pj.z), G.periodic[2], K.L[2], K.halfL[2]) : Real(0);
                Real r2 = dist2<Real, DIM>(dx, dy, dz);
                if (!(r2 < K.kh2)) continue;
                const bool fluid_j = pj.w > Real(0);
                const typename V4<Real>::T qj = Q[j];
                const Real mj = fabs(pj.w);
                const Real q = sqrt(r2) * K.inv_h;
                const Real Gk = K.gfac * kernel_f<Real, KERNEL>(q);  // grad_i W = Gk (x_i - x_j)
                const Real vx = qi.x - qj.x, vy = qi.y - qj.y, vz = DIM == 3 ? qi.z - qj.z : Real(0);
                Real coef = pri + R[j];
                const Real rhobar = Real(0.5) * (qi.w + qj.w);
                if (flags & F_AV) {
                    const Real vdotr = vx * dx + vy * dy + (DIM == 3 ? vz * dz : Real(0));
                    if (vdotr < Real(0)) {
                        const Real mu = K.h * vdotr / (r2 + K.av_h2);
                        coef -= K.alpha_c0 * mu / rhobar;
                    }
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
        for (int d = 0; d < DIM; ++d) a[d] += C.g[d];
        double u[3] = {0, 0, 0};
        double u2 = 0, a2 = 0;
        for (int d = 0; d < DIM; ++d) {
            S.a[d][i] = a[d];
            S.xs[d][i] = xs[d];
            u[d] = S.u[d][i];
            if (kick) {
                u[d] += 0.5 * dt * a[d];
                S.u[d][i] = u[d];
            }
            u2 += u[d] * u[d];
            a2 += a[d] * a[d];
            if (!isfinite(u[d]) || !isfinite(S.x[d][i])) bad = 1;
        }
        if (!isfinite(S.rho[i]) || !isfinite(a2)) bad = 1;
        const double m = S.m[i];
        d_px += m * u[0];
        d_py += m * u[1];
        d_pz += m * u[2];
        d_ke += 0.5 * m * u2;
        d_u2 = fmax(d_u2, u2);
        d_a2 = fmax(d_a2, a2);
    }

    // ---- block reduction (fixed tree order: deterministic)
    constexpr int NV = 7;  // px py pz ke u2max a2max bad
    __shared__ double red[PAIR_THREADS / 32][NV];
    __shared__ bool is_last;
    double v[NV] = {d_px, d_py, d_pz, d_ke, d_u2, d_a2, (double)bad};
    auto is_max = [](int k) { return k >= 4; };
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double y = __shfl_down_sync(0xffffffffu, v[k], o);
            v[k] = is_max(k) ? fmax(v[k], y) : v[k] + y;
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) red[warp][k] = v[k];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double t = red[0][k];
            for (int w = 1; w < PAIR_THREADS / 32; ++w) t = is_max(k) ? fmax(t, red[w][k]) : t + red[w][k];
            partials[(size_t)blockIdx.x * PARTIAL_STRIDE + k] = t;
        }
        __threadfence();
        unsigned t = atomicAdd(&ctl->ticket, 1u);
        is_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    // ---- last block: reduce the partials (this pass: 0..6, density pass: 10..12)
    constexpr int NT = 10;
    double w[NT];
#pragma unroll
    for (int k = 0; k < NT; ++k) w[k] = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
        const volatile double* p = partials + (size_t)b * PARTIAL_STRIDE;
#pragma unroll
        for (int k = 0; k < NV; ++k) w[k] = is_max(k) ? fmax(w[k], p[k]) : w[k] + p[k];
#pragma unroll
        for (int k = 0; k < 3; ++k) w[NV + k] += p[10 + k];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int k = 0; k < NT; ++k) {
            double y = __shfl_down_sync(0xffffffffu, w[k], o);
            w[k] = (k >= 4 && k < NV) ? fmax(w[k], y) : w[k] + y;
        }
    }
    __shared__ double red2[PAIR_THREADS / 32][NT];
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < NT; ++k) red2[warp][k] = w[k];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double out[NT];
#pragma unroll
        for (int k = 0; k < NT; ++k) {
            double t = red2[0][k];
            for (int ww = 1; ww < PAIR_THREADS / 32; ++ww)
                t = (k >= 4 && k < NV) ? fmax(t, red2[ww][k]) : t + red2[ww][k];
            out[k] = t;
        }
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
        rec[8] = out[7];
        rec[9] = out[8];
        rec[10] = (double)ctl->step;
        rec[11] = (double)ctl->outside;
        rec[12] = out[9];
        if (out[6] != 0.0) ctl->status |= ST_NONFINITE;
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
    k_density<Real, DIM, KERNEL><<<L.grid, PAIR_THREADS, 0, st>>>(
        (const V*)L.P, (V*)L.Q, (Real*)L.R, L.skeys, L.off, L.n, L.G, K, L.C, L.S, L.ctl, L.kick,
        L.partials);
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
