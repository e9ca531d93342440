// Pair loops of one right-hand-side evaluation over the cell-sorted particles
// (Sec. 3.2 groups; per-destination loop of Sec. 3.4), as kernel templates:
//  - the density pass: summation density, Eq. (2), or the continuity rate,
//    Eq. (continuity:sph), with the position-like density advance, then the EOS;
//  - the momentum pass: pressure Eq. (mom:sph:press), laminar viscosity
//    Eq. (mom:sph:visc), Monaghan artificial viscosity, XSPH and the body force of
//    Eq. (mom:sph), with the corrector half-kick of Sec. 2.1 and the FP64 diagnostics.
//
// Work decomposition: the density pass gives one thread to each destination, walks the
// 3^(d-1) contiguous source runs of its stencil (a tight load-test loop) and records the
// accepted sources in an interleaved neighbour list (nl[k * n + i]: lanes of a warp read
// consecutive words); its density sum and the whole momentum pass then loop over that
// list with no predicate and little divergence. In the momentum pass a group of T lanes
// (T = 1, 2, 4 or 8, the tile shape the autotuner picks) shares one destination; each
// lane keeps compensated partial sums and a fixed shuffle tree combines them, so results
// are deterministic.
#pragma once

#include "sph_device.cuh"
#include "sph_launch.h"
#include "step_impl.cuh"
#include "reduce_impl.cuh"

namespace sph {

constexpr int PAIR_THREADS = 128;

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

// The T lanes of one destination inside a warp.
template <int T>
struct Group {
    int t;          // lane within the group
    int shift;      // first warp lane of the group
    unsigned mask;  // warp lanes of the group
    __device__ __forceinline__ Group() {
        const int lane = threadIdx.x & 31;
        t = lane & (T - 1);
        shift = lane - t;
        mask = (T == 32) ? 0xffffffffu : (((1u << T) - 1u) << shift);
    }
    __device__ __forceinline__ unsigned ballot(bool p) const {
        const unsigned b = __ballot_sync(mask, p);
        return T == 32 ? b : ((b >> shift) & ((1u << T) - 1u));
    }
    __device__ __forceinline__ void sync() const { __syncwarp(mask); }
    template <class V>
    __device__ __forceinline__ V down(V v, int o) const { return __shfl_down_sync(mask, v, o, T); }
};

// Combines the lanes' compensated partial sums into lane 0 (fixed order).
template <class Real, int T>
__device__ __forceinline__ void group_reduce(Acc<Real>& a, const Group<T>& g) {
#pragma unroll
    for (int o = T / 2; o > 0; o >>= 1) {
        const Real s2 = g.down(a.s, o);
        const Real c2 = g.down(a.c, o);
        a.add(s2);
        a.c += c2;
    }
}

// Separation of i and j with the neighbour predicate's exact arithmetic.
template <class Real, int DIM>
__device__ __forceinline__ Real separation(const typename V4<Real>::T& pi,
                                           const typename V4<Real>::T& pj, const Grid& G,
                                           const PairConst<Real>& K, Real& dx, Real& dy, Real& dz) {
    dx = min_image(rn_sub(pi.x, pj.x), G.periodic[0], K.L[0], K.halfL[0]);
    dy = min_image(rn_sub(pi.y, pj.y), G.periodic[1], K.L[1], K.halfL[1]);
    dz = DIM == 3 ? min_image(rn_sub(pi.z, pj.z), G.periodic[2], K.L[2], K.halfL[2]) : Real(0);
    return dist2<Real, DIM>(dx, dy, dz);
}

// Block sum of 3 counters into pd[blockIdx.x * 4 + k] (fixed tree order).
__device__ __forceinline__ void block_counts(double c0, double c1, double c2, double* pd) {
    __shared__ double red[PAIR_THREADS / 32][3];
    double v[3] = {c0, c1, c2};
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int k = 0; k < 3; ++k) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < 3; ++k) red[warp][k] = v[k];
    __syncthreads();
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            double t = red[0][k];
            for (int w = 1; w < PAIR_THREADS / 32; ++w) t += red[w][k];
            pd[(size_t)blockIdx.x * 4 + k] = t;
        }
}

// ---------------------------------------------------------------- density pass
// A group of T lanes per destination (T = 1, 2, 4 or 8). (1) Neighbour scan: the 3^(d-1)
// contiguous source runs of the destination's stencil, T candidates at a time (lane t
// takes the t-th), the exact neighbour predicate, and the accepted sources appended to
// the interleaved neighbour list nl[k * n + i] (k < maxn; cnt[i] entries) in candidate
// order: a ballot over the group gives each accepted lane its slot, so the list is the
// same for every T. Continuity mode lists interacting sources only (a wall destination
// takes fluid sources); summation mode lists every neighbour. (2) The density group
// over the list, lane t taking every T-th entry with compensated partial sums combined
// by a fixed shuffle tree:
//  summation (Eq. 2): rho_i = sum_j m_j W_ij, self term included;
//  continuity (Eq. continuity:sph): arho_i = sum_j m_j v_ij . grad_i W_ij and, inside a
//    step, rho_i += dt arho_i (density advanced like the positions, Sec. 2.1 reading).
// Then p from the Tait EOS in FP64 and the shadow rho, p / rho^2. Counts interacting pairs
// (not both walls), candidates and the interacting pairs with a wall destination. A list
// overflow raises ST_CAPACITY (the evaluation is then invalid and the step reports it).
struct DensityCounts {
    double pairs, cand, wall;
    int overflow;
};

template <int T>
__device__ __forceinline__ uint32_t group_sum_u32(uint32_t v, const Group<T>& g) {
#pragma unroll
    for (int o = T / 2; o > 0; o >>= 1) v += g.down(v, o);
    return v;
}

// Density pass for destination i (cell key `key`, cell table `off` of its grid), shared by
// the T lanes of group g (lane 0 finishes).
template <class Real, int DIM, int KERNEL, int T>
__device__ __forceinline__ void density_dest(int i, const Group<T>& g, uint32_t key,
                                             const typename V4<Real>::T* __restrict__ P,
                                             typename V4<Real>::T* __restrict__ Q,
                                             Real* __restrict__ R, const uint32_t* __restrict__ off,
                                             int n, const Grid& G, const PairConst<Real>& K,
                                             const StepConst& C, const ParticleSet& S, double dt,
                                             int kick, uint32_t* __restrict__ nl,
                                             uint32_t* __restrict__ cnt, int maxn,
                                             DensityCounts& dc, uint32_t* npairs_out,
                                             uint32_t* ncand_out) {
    const bool summation = !(K.flags & F_CONTINUITY);
    const typename V4<Real>::T pi = P[i];
    const bool fluid_i = pi.w > Real(0);
    int cx, cy, cz;
    cell_of_key(G, key, cx, cy, cz);
    uint32_t k = 0, npairs = 0, ncand = 0;
    const unsigned below = (1u << g.t) - 1u;
    for_each_run<DIM>(G, off, cx, cy, cz, [&](uint32_t jb, uint32_t je) {
#pragma unroll 2
        for (uint32_t c = jb; c < je; c += T) {
            const uint32_t j = c + g.t;
            bool listed = false;
            if (j < je && (int)j != i) {
                ++ncand;
                const typename V4<Real>::T pj = P[j];
                Real dx, dy, dz;
                const Real r2 = separation<Real, DIM>(pi, pj, G, K, dx, dy, dz);
                if (r2 < K.kh2) {
                    const bool interacting = fluid_i || pj.w > Real(0);
                    listed = interacting || summation;
                    npairs += interacting ? 1u : 0u;
                }
            }
            if (T == 1) {
                if (listed) {
                    if (k < (uint32_t)maxn) nl[(size_t)k * n + i] = j;
                    ++k;
                }
            } else {
                const unsigned m = g.ballot(listed);
                if (listed) {
                    const uint32_t pos = k + __popc(m & below);
                    if (pos < (uint32_t)maxn) nl[(size_t)pos * n + i] = j;
                }
                k += __popc(m);
            }
        }
    });
    if (k > (uint32_t)maxn) {
        dc.overflow = 1;
        k = maxn;
    }
    if (g.t == 0) cnt[i] = k;
    g.sync();  // the list entries of the other lanes are visible from here on
    Acc<Real> sum;
    sum.zero();
    const typename V4<Real>::T qi = Q[i];
    for (uint32_t kk = g.t; kk < k; kk += T) {
        const uint32_t j = nl[(size_t)kk * n + i];
        const typename V4<Real>::T pj = P[j];
        Real dx, dy, dz;
        const Real r2 = separation<Real, DIM>(pi, pj, G, K, dx, dy, dz);
        const Real q = sqrt(r2) * K.inv_h;
        if (summation) {
            sum.add(fabs(pj.w) * K.wfac * kernel_w<Real, KERNEL>(q));
        } else {
            const typename V4<Real>::T qj = Q[j];
            const Real Gk = K.gfac * kernel_f<Real, KERNEL>(q);
            const Real vdotr = (qi.x - qj.x) * dx + (qi.y - qj.y) * dy +
                               (DIM == 3 ? (qi.z - qj.z) * dz : Real(0));
            sum.add(fabs(pj.w) * Gk * vdotr);
        }
    }
    if (T > 1) group_reduce<Real, T>(sum, g);
    dc.pairs += (double)npairs;
    dc.cand += (double)ncand;
    if (!fluid_i) dc.wall += (double)npairs;
    if (npairs_out) {
        const uint32_t np = group_sum_u32<T>(npairs, g), nc = group_sum_u32<T>(ncand, g);
        if (g.t == 0) {
            *npairs_out = np;
            *ncand_out = nc;
        }
    }
    if (g.t != 0) return;
    double rho;
    if (summation) {
        rho = sum.value() + (double)(fabs(pi.w) * K.wfac * kernel_w<Real, KERNEL>(Real(0)));
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
}

// Density pass over all destinations; each finds its instance's constants in the table
// (one entry for a single problem). Single problems accumulate block counts in pd; batches
// store per-particle counts in pcount for the per-instance reduction.
template <class Real, int DIM, int KERNEL, int T>
__global__ void __launch_bounds__(PAIR_THREADS, 6)
k_density(const typename V4<Real>::T* __restrict__ P, typename V4<Real>::T* __restrict__ Q,
          Real* __restrict__ R, const uint32_t* __restrict__ skeys, const uint32_t* __restrict__ off,
          int n, const Inst<Real>* __restrict__ tab, const uint32_t* __restrict__ cell_bounds,
          int ninst, const double* __restrict__ idt, ParticleSet S, Control* ctl, int kick,
          uint32_t* __restrict__ nl, uint32_t* __restrict__ cnt, int maxn,
          double* __restrict__ pd, uint32_t* __restrict__ pcount) {
    if (ctl->status) return;
    const Group<T> g;
    DensityCounts dc{0, 0, 0, 0};
    const int groups = gridDim.x * (PAIR_THREADS / T);
    for (int i = (blockIdx.x * PAIR_THREADS + threadIdx.x) / T; i < n; i += groups) {
        const uint32_t key = skeys[i];
        const int inst = find_instance(cell_bounds, ninst, key);
        const Inst<Real>& I = tab[inst];
        density_dest<Real, DIM, KERNEL, T>(i, g, key - I.cell_base, P, Q, R, off + I.cell_base, n,
                                           I.G, I.K, I.C, S, idt[inst], kick, nl, cnt, maxn, dc,
                                           pcount ? pcount + 2 * (size_t)i : nullptr,
                                           pcount ? pcount + 2 * (size_t)i + 1 : nullptr);
    }
    if (dc.overflow) atomicOr(&ctl->status, ST_CAPACITY);
    if (pd) block_counts(dc.pairs, dc.cand, dc.wall, pd);
}

// ------------------------------------------------------------- momentum pass
// Fluid destinations only (walls are static), over the neighbour list of the density
// pass: S lanes per destination take every S-th list entry (the tile shape the autotuner
// picks) and combine their compensated partial sums with a fixed shuffle tree. Then the
// corrector half-kick u^{n+1} = u^{n+1/2} + dt/2 a^{n+1} inside a step and the FP64
// diagnostics. The last block to finish reduces the block partials of both passes in a
// fixed order (deterministic) and writes the record, history entry, next dt and status.
struct MomDiag {
    double px, py, pz, ke, u2, a2;
    int bad;
};

// Momentum pass for destination i, shared by the T lanes of group g (lane 0 finishes).
template <class Real, int DIM, int KERNEL, int T>
__device__ __forceinline__ void momentum_dest(int i, const Group<T>& g,
                                              const typename V4<Real>::T* __restrict__ P,
                                              const typename V4<Real>::T* __restrict__ Q,
                                              const Real* __restrict__ R, int n,
                                              const Grid& G, const PairConst<Real>& K,
                                              const StepConst& C, const ParticleSet& S, double dt,
                                              int kick, const uint32_t* __restrict__ nl,
                                              const uint32_t* __restrict__ cnt, MomDiag& md) {
    const int flags = K.flags;
    const typename V4<Real>::T pi = P[i];
    const bool fluid_i = pi.w > Real(0);
    if (!fluid_i) {  // walls: no momentum equation, static
        if (g.t == 0) {
            for (int d = 0; d < DIM; ++d) {
                S.a[d][i] = 0.0;
                S.xs[d][i] = 0.0;
            }
            if (!isfinite(S.rho[i])) md.bad = 1;
        }
        return;
    }
    const typename V4<Real>::T qi = Q[i];
    const Real pri = R[i];
    Acc<Real> ax, ay, az, sx, sy, sz;
    ax.zero(); ay.zero(); az.zero(); sx.zero(); sy.zero(); sz.zero();
    const uint32_t ni = cnt[i];
    for (uint32_t kk = g.t; kk < ni; kk += T) {
        const uint32_t j = nl[(size_t)kk * n + i];
        const typename V4<Real>::T pj = P[j];
        Real dx, dy, dz;
        const Real r2 = separation<Real, DIM>(pi, pj, G, K, dx, dy, dz);
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
        if ((flags & F_XSPH) && pj.w > Real(0)) {
            const Real fx = K.xsph * mj / rhobar * (K.wfac * kernel_w<Real, KERNEL>(q));
            sx.add(-fx * vx);
            sy.add(-fx * vy);
            if (DIM == 3) sz.add(-fx * vz);
        }
    }
    if (T > 1) {
        group_reduce<Real, T>(ax, g);
        group_reduce<Real, T>(ay, g);
        if (DIM == 3) group_reduce<Real, T>(az, g);
        if (flags & F_XSPH) {
            group_reduce<Real, T>(sx, g);
            group_reduce<Real, T>(sy, g);
            if (DIM == 3) group_reduce<Real, T>(sz, g);
        }
    }
    if (g.t == 0) {  // epilogue: FP64 rates, corrector half-kick, diagnostics
        double a[3] = {ax.value(), ay.value(), az.value()};
        double xs[3] = {sx.value(), sy.value(), sz.value()};
        double u[3] = {0, 0, 0};
        double u2 = 0, a2 = 0;
        for (int d = 0; d < DIM; ++d) {
            a[d] += C.g[d];
            S.a[d][i] = a[d];
            S.xs[d][i] = xs[d];
            u[d] = S.u[d][i];
            if (kick) {
                u[d] += 0.5 * dt * a[d];
                S.u[d][i] = u[d];
            }
            u2 += u[d] * u[d];
            a2 += a[d] * a[d];
            if (!isfinite(u[d]) || !isfinite(S.x[d][i])) md.bad = 1;
        }
        if (!isfinite(S.rho[i]) || !isfinite(a2)) md.bad = 1;
        const double m = S.m[i];
        md.px += m * u[0];
        md.py += m * u[1];
        md.pz += m * u[2];
        md.ke += 0.5 * m * u2;
        md.u2 = fmax(md.u2, u2);
        md.a2 = fmax(md.a2, a2);
    }
}

// Momentum pass over all destinations (instance constants from the table). With
// finalize (single problems) the block partials of both passes are reduced by the last
// block, which writes the record, the history entry, the next dt and the status.
template <class Real, int DIM, int KERNEL, int T>
__global__ void __launch_bounds__(PAIR_THREADS, 5)
k_momentum(const typename V4<Real>::T* __restrict__ P, const typename V4<Real>::T* __restrict__ Q,
           const Real* __restrict__ R, const uint32_t* __restrict__ skeys, int n,
           const Inst<Real>* __restrict__ tab, const uint32_t* __restrict__ cell_bounds, int ninst,
           double* __restrict__ idt, ParticleSet S, Control* ctl, int kick,
           const uint32_t* __restrict__ nl, const uint32_t* __restrict__ cnt,
           double* __restrict__ pm, const double* __restrict__ pd, int density_blocks,
           double* __restrict__ history, int finalize) {
    __shared__ double red[PAIR_THREADS / 32][10];
    __shared__ bool is_last;
    if (ctl->status) return;
    const Group<T> g;
    const double dt = idt[0];
    MomDiag md{0, 0, 0, 0, 0, 0, 0};
    const int groups = gridDim.x * (PAIR_THREADS / T);
    for (int i = (blockIdx.x * PAIR_THREADS + threadIdx.x) / T; i < n; i += groups) {
        const int inst = find_instance(cell_bounds, ninst, skeys[i]);
        const Inst<Real>& I = tab[inst];
        momentum_dest<Real, DIM, KERNEL, T>(i, g, P, Q, R, n, I.G, I.K, I.C, S, idt[inst], kick,
                                            nl, cnt, md);
    }
    if (!finalize) return;
    const StepConst& C = tab[0].C;
    double d_px = md.px, d_py = md.py, d_pz = md.pz, d_ke = md.ke, d_u2 = md.u2, d_a2 = md.a2;
    int bad = md.bad;

    // ---- block reduction (fixed tree order: deterministic)
    constexpr int NV = 7;  // px py pz ke u2max a2max bad
    double v[NV] = {d_px, d_py, d_pz, d_ke, d_u2, d_a2, (double)bad};
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            const double y = __shfl_down_sync(0xffffffffu, v[k], o);
            v[k] = k >= 4 ? fmax(v[k], y) : v[k] + y;
        }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) red[warp][k] = v[k];
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double t = red[0][k];
            for (int w = 1; w < PAIR_THREADS / 32; ++w) t = k >= 4 ? fmax(t, red[w][k]) : t + red[w][k];
            pm[(size_t)blockIdx.x * 8 + k] = t;
        }
        __threadfence();
        const unsigned t = atomicAdd(&ctl->ticket, 1u);
        is_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    // ---- last block: momentum partials (7) and density-pass counts (3), fixed order
    constexpr int NT = 10;
    double w[NT];
#pragma unroll
    for (int k = 0; k < NT; ++k) w[k] = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += PAIR_THREADS) {
        const volatile double* p = pm + (size_t)b * 8;
#pragma unroll
        for (int k = 0; k < NV; ++k) w[k] = k >= 4 ? fmax(w[k], p[k]) : w[k] + p[k];
    }
    for (int b = threadIdx.x; b < density_blocks; b += PAIR_THREADS) {
        const volatile double* p = pd + (size_t)b * 4;
#pragma unroll
        for (int k = 0; k < 3; ++k) w[NV + k] += p[k];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int k = 0; k < NT; ++k) {
            const double y = __shfl_down_sync(0xffffffffu, w[k], o);
            w[k] = (k >= 4 && k < NV) ? fmax(w[k], y) : w[k] + y;
        }
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NT; ++k) red[warp][k] = w[k];
    __syncthreads();
    if (threadIdx.x == 0) {
        double out[NT];
#pragma unroll
        for (int k = 0; k < NT; ++k) {
            double t = red[0][k];
            for (int ww = 1; ww < PAIR_THREADS / 32; ++ww)
                t = (k >= 4 && k < NV) ? fmax(t, red[ww][k]) : t + red[ww][k];
            out[k] = t;
        }
        ctl->ticket = 0;
        finish_single(ctl, history, C, dt, kick, out);
    }
}

// ---------------------------------------------------------------- launchers
template <class Real, int DIM, int KERNEL, int T>
int density_bps() {
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_density<Real, DIM, KERNEL, T>, PAIR_THREADS, 0);
    return b > 0 ? b : 1;
}

template <class Real, int DIM, int KERNEL, int T>
int momentum_bps() {
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_momentum<Real, DIM, KERNEL, T>, PAIR_THREADS, 0);
    return b > 0 ? b : 1;
}

template <class Real, int DIM, int KERNEL, int T>
void launch_density_t(const StepLaunch& L, cudaStream_t st) {
    using V = typename V4<Real>::T;
    k_density<Real, DIM, KERNEL, T><<<L.grid_d, PAIR_THREADS, 0, st>>>(
        (const V*)L.P, (V*)L.Q, (Real*)L.R, L.skeys, L.off, L.n, (const Inst<Real>*)L.tab,
        L.cell_bounds, L.ninst, L.idt, L.S, L.ctl, L.kick, L.nl, L.cnt, L.maxn,
        L.finalize ? L.pd : nullptr, L.finalize ? nullptr : L.pcount);
}

template <class Real, int DIM, int KERNEL, int T>
void launch_momentum_t(const StepLaunch& L, cudaStream_t st) {
    using V = typename V4<Real>::T;
    k_momentum<Real, DIM, KERNEL, T><<<L.grid_m, PAIR_THREADS, 0, st>>>(
        (const V*)L.P, (const V*)L.Q, (const Real*)L.R, L.skeys, L.n, (const Inst<Real>*)L.tab,
        L.cell_bounds, L.ninst, L.idt, L.S, L.ctl, L.kick, L.nl, L.cnt, L.pm, L.pd, L.grid_d,
        L.history, L.finalize);
}

// One precision's dispatch over (dim, kernel, group size).
template <class Real>
struct PairDispatch {
    template <int T>
    static int bps_t(int pass, int dim, int kernel) {
        const int sel = (dim == 3 ? 2 : 0) + (kernel == WENDLAND_C2 ? 1 : 0);
        switch (sel) {
            case 0: return pass ? momentum_bps<Real, 2, QUINTIC, T>() : density_bps<Real, 2, QUINTIC, T>();
            case 1: return pass ? momentum_bps<Real, 2, WENDLAND_C2, T>() : density_bps<Real, 2, WENDLAND_C2, T>();
            case 2: return pass ? momentum_bps<Real, 3, QUINTIC, T>() : density_bps<Real, 3, QUINTIC, T>();
            default: return pass ? momentum_bps<Real, 3, WENDLAND_C2, T>() : density_bps<Real, 3, WENDLAND_C2, T>();
        }
    }
    template <int T>
    static void density_t(const StepLaunch& L, cudaStream_t st) {
        const int sel = (L.dim == 3 ? 2 : 0) + (L.kernel == WENDLAND_C2 ? 1 : 0);
        switch (sel) {
            case 0: launch_density_t<Real, 2, QUINTIC, T>(L, st); break;
            case 1: launch_density_t<Real, 2, WENDLAND_C2, T>(L, st); break;
            case 2: launch_density_t<Real, 3, QUINTIC, T>(L, st); break;
            default: launch_density_t<Real, 3, WENDLAND_C2, T>(L, st); break;
        }
    }
    template <int T>
    static void momentum_t(const StepLaunch& L, cudaStream_t st) {
        const int sel = (L.dim == 3 ? 2 : 0) + (L.kernel == WENDLAND_C2 ? 1 : 0);
        switch (sel) {
            case 0: launch_momentum_t<Real, 2, QUINTIC, T>(L, st); break;
            case 1: launch_momentum_t<Real, 2, WENDLAND_C2, T>(L, st); break;
            case 2: launch_momentum_t<Real, 3, QUINTIC, T>(L, st); break;
            default: launch_momentum_t<Real, 3, WENDLAND_C2, T>(L, st); break;
        }
    }
};

}  // namespace sph
