// Persistent step: the whole time step (Sec. 2.1 predictor-corrector with the Sec. 2.2
// neighbour build and the Sec. 3.4 pair loops) as ONE cooperative launch. Every block
// stays resident for the step and walks each phase with a grid-stride loop; the phases
// are separated by a grid-wide barrier:
//   drift + cell keys | radix sort (histogram | digit scan | scatter, per 8-bit pass) |
//   reorder + predictor kick + EOS shadow, and the cell table | density pass |
//   [solid-wall pressure] | momentum pass + corrector kick | diagnostics, next dt (for a
//   batch per instance, in the two stages of the batch kernels with a barrier between).
// The per-particle and per-tile bodies are the ones of the per-phase kernels, so both
// forms compute the same step; a small problem saves the launch gaps between phases.
//
// The barrier spins on a generation counter in the control block with a time limit:
// a block that waits longer raises ST_TIMEOUT and leaves, and the others leave at their
// next barrier (they also watch the status word), so no wait is unbounded. A limit of 0
// lets no block wait at all (the first barrier of a multi-block grid then fails).
#pragma once

#include "pairs_impl.cuh"
#include "fused_units.h"
#include "batch_impl.cuh"
#include "sort_impl.cuh"
#include "step_impl.cuh"
#include "walls_impl.cuh"

namespace sph {

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid-wide barrier (all blocks co-resident: cooperative launch). Returns false, in every
// thread of the block, if the step must stop: the wait ran out (ST_TIMEOUT raised here)
// or a status bit is set.
__device__ __forceinline__ bool grid_sync(Control* ctl, unsigned long long limit_ns) {
    __syncthreads();
    int ok = 1;
    if (threadIdx.x == 0) {
        volatile unsigned* gen = &ctl->bar_gen;
        volatile unsigned* status = &ctl->status;
        const unsigned g = *gen;
        __threadfence();
        const unsigned arrived = atomicAdd(&ctl->bar_count, 1u);
        if (arrived == gridDim.x - 1) {
            atomicExch(&ctl->bar_count, 0u);
            __threadfence();
            atomicAdd(&ctl->bar_gen, 1u);
        } else {
            const unsigned long long t0 = global_ns();
            while (*gen == g) {
                if (limit_ns == 0 || (*status & ST_TIMEOUT) || global_ns() - t0 > limit_ns) {
                    atomicOr(&ctl->status, ST_TIMEOUT);
                    ok = 0;
                    break;
                }
                __nanosleep(40);
            }
        }
        __threadfence();
        if (*status) ok = 0;
    }
    return __syncthreads_and(ok) != 0;
}

// FP32: 3 blocks of 256 per SM (80 registers; the pair phases are latency-bound and gain
// from the extra warps), FP64: 2.
template <class Real, int DIM, int KERNEL, int T>
__global__ void __launch_bounds__(FUSED_THREADS, sizeof(Real) == 4 ? 3 : 2) k_step_fused(const FusedLaunch F) {
    using V = typename V4<Real>::T;
    __shared__ union {
        uint32_t h[4][RADIX];
        OnesweepSmem os;
        DensitySmem<Real, T == 1 ? 1 : FUSED_THREADS / T> dens;
        MomSmem<Real, T == 1 ? 1 : FUSED_THREADS / T> mom;
        double bred[FUSED_THREADS / 32][10];
        struct {
            MomDiag mred[FUSED_THREADS / 32];
            unsigned long long cred[FUSED_THREADS / 32][3];
        };
    } sm;
    __shared__ int tile_s;
    const StepLaunch& L = F.L;
    Control* ctl = L.ctl;
    if (ctl->status) return;
    const Inst<Real>* __restrict__ tab = (const Inst<Real>*)L.tab;
    const int nb = gridDim.x;
    const int tid = blockIdx.x * FUSED_THREADS + threadIdx.x, nthreads = nb * FUSED_THREADS;
    const bool stamp = blockIdx.x == 0 && threadIdx.x == 0;
    V* P = (V*)L.P;
    V* Q = (V*)L.Q;
    Real* R = (Real*)L.R;
    F4* E = (F4*)L.E;  // FP32 pair loops: position residuals (null in FP64 mode)
    uint32_t* ghist = F.work;
    uint32_t* counters = F.work + 4 * RADIX;
    uint32_t* status = counters + 32;
    if (stamp) ctl->stamp[0] = global_ns();

    // ---- drift of the fluid (predictor half-kick folded in) + cell keys + digit histograms
    {
        for (int p = 0; p < F.passes; ++p) sm.h[p][threadIdx.x] = 0;
        __syncthreads();
        unsigned outside = 0;
        for (int base = blockIdx.x * FUSED_THREADS; base < L.n; base += nthreads) {
            const int i = base + threadIdx.x;
            const bool valid = i < L.n;
            uint32_t key = 0;
            if (valid) {
                const int inst = find_instance(L.id_bounds, L.ninst, L.Sin.tag[i] & ID_MASK);
                const Inst<Real>& I = tab[inst];
                int clamped = 0;
                key = I.cell_base + drift_key_one(L.Sin, i, I.G, I.C, L.idt[inst], 1, clamped);
                F.keys[0][i] = key;
                outside += clamped;
            }
            digit_hist_add(key, valid, F.passes, sm.h);
        }
        for (int o = 16; o > 0; o >>= 1) outside += __shfl_down_sync(0xffffffffu, outside, o);
        if ((threadIdx.x & 31) == 0 && outside) atomicAdd(&ctl->outside, outside);
        __syncthreads();
        for (int p = 0; p < F.passes; ++p) {
            const uint32_t v = sm.h[p][threadIdx.x];
            if (v) atomicAdd(&ghist[p * RADIX + threadIdx.x], v);
        }
    }
    if (!grid_sync(ctl, F.wait_ns)) return;
    if (stamp) ctl->stamp[1] = global_ns();

    // ---- stable LSD radix sort of (key, index): one-sweep passes, tiles taken in order
    int cur = 0;
    for (int p = 0; p < F.passes; ++p) {
        for (;;) {
            if (threadIdx.x == 0) tile_s = (int)atomicAdd(&counters[p], 1u);
            __syncthreads();
            const int t = tile_s;
            if (t >= F.ntiles) break;
            const uint32_t* vin = p ? F.vals[cur] : nullptr;
            uint32_t* st_p = status + (size_t)p * F.ntiles * RADIX;
            switch (onesweep_items(L.n)) {
                case 4:
                    radix_onesweep_tile<4>(F.keys[cur], vin, F.keys[cur ^ 1], F.vals[cur ^ 1], L.n,
                                           8 * p, ghist + p * RADIX, st_p, t, sm.os, &ctl->status,
                                           F.wait_ns);
                    break;
                default:
                    radix_onesweep_tile<8>(F.keys[cur], vin, F.keys[cur ^ 1], F.vals[cur ^ 1], L.n,
                                           8 * p, ghist + p * RADIX, st_p, t, sm.os, &ctl->status,
                                           F.wait_ns);
                    break;
            }
            __syncthreads();
        }
        if (!grid_sync(ctl, F.wait_ns)) return;
        cur ^= 1;
    }
    if (stamp) ctl->stamp[2] = global_ns();
    const uint32_t* __restrict__ skeys = F.keys[cur];
    const uint32_t* __restrict__ perm = F.vals[cur];

    // ---- gather into cell order (predictor kick, shadow) and the cell table
    for (int k = tid; k < L.n; k += nthreads) {
        const int inst = find_instance(L.cell_bounds, L.ninst, skeys[k]);
        reorder_one<Real>(L.Sin, L.S, k, (int)perm[k], L.dim, L.idt[inst], 1, 0, P, Q, E, L.edac);
    }
    for (int c = tid; c <= F.ncells; c += nthreads)
        F.off[c] = cell_offset_near(skeys, L.n, (uint32_t)c, F.off[c]);
    if (!grid_sync(ctl, F.wait_ns)) return;
    if (stamp) ctl->stamp[3] = global_ns();

    // ---- density pass (T lanes per destination, compact FP64 epilogue)
    {
        DensityCounts dc{0ull, 0ull, 0ull, 0};
        density_tiles<Real, DIM, KERNEL, T, FUSED_THREADS>(
            blockIdx.x, nb, P, Q, R, E, skeys, F.off, L.n, tab, L.cell_bounds, L.ninst, L.idt, L.S, 1,
            L.nl, L.cnt, L.maxn, L.finalize ? nullptr : L.pcount, dc, sm.dens);
        if (dc.overflow) atomicOr(&ctl->status, ST_CAPACITY);
        if (L.finalize) block_counts<FUSED_THREADS>(dc, F.part + (size_t)blockIdx.x * FUSED_PART + 8, sm.cred);
    }
    if (!grid_sync(ctl, F.wait_ns)) return;

    // ---- solid-wall pressure of the wall particles from their fluid neighbours
    if (F.wall_pass) {
        wall_pressure_range<Real, DIM, KERNEL, FUSED_THREADS>(blockIdx.x, nb, P, Q, R, skeys, L.n, tab,
                                                              L.cell_bounds, L.ninst, L.S, L.nl, L.cnt);
        if (!grid_sync(ctl, F.wait_ns)) return;
    }
    if (stamp) ctl->stamp[4] = global_ns();

    // ---- momentum pass (T lanes per destination) + corrector kick; the sort workspace is
    // no longer read in this step and is zeroed for the next one
    for (int w = tid; w < F.work_words; w += nthreads) F.work[w] = 0u;
    {
        MomDiag md{0, 0, 0, 0, 0ull, 0ull, 0u};
        momentum_tiles<Real, DIM, KERNEL, T, FUSED_THREADS>(blockIdx.x, nb, P, Q, R, E, skeys, L.n, tab,
                                                            L.cell_bounds, L.ninst, L.idt, L.S, 1,
                                                            L.nl, L.cnt, md, sm.mom);
        if (L.finalize)
            block_mom_diag<(FUSED_THREADS / T + 31) / 32>(md, F.part + (size_t)blockIdx.x * FUSED_PART,
                                                         sm.mred);
    }
    if (!grid_sync(ctl, F.wait_ns)) return;
    if (stamp) ctl->stamp[5] = global_ns();

    // ---- diagnostics, time and next dt
    if (L.finalize) {
        if (blockIdx.x != 0) return;
        double out[10];
        reduce_partials<FUSED_THREADS>(F.part, FUSED_PART, nb, F.part + 8, FUSED_PART, nb, out,
                                       sm.mred, sm.cred);
        if (threadIdx.x == 0) {
            finish_single(ctl, L.history, tab[0].C, L.idt[0], 1, out);
            ctl->outside = 0;
            ctl->stamp[6] = global_ns();
        }
    } else {
        // the two stages of the batch kernels (same chunks, same fixed-order combination)
        // with a barrier between them, so every block takes part in the first
        for (int w = blockIdx.x; w < L.ninst * BATCH_SPLIT; w += nb)
            batch_chunk_partials<Real, FUSED_THREADS>(L.S, L.pcount, F.off, tab[w / BATCH_SPLIT],
                                                      w / BATCH_SPLIT, w % BATCH_SPLIT, L.dim, L.bpart,
                                                      sm.bred);
        if (!grid_sync(ctl, F.wait_ns)) return;
        for (int inst = (blockIdx.x * FUSED_THREADS + threadIdx.x) >> 5; inst < L.ninst;
             inst += nb * (FUSED_THREADS / 32))
            batch_finish_warp<Real>(tab[inst], inst, L.bpart, L.idt, L.it, L.irec, 1, ctl);
        if (stamp) {
            ctl->outside = 0;
            ctl->stamp[6] = global_ns();
        }
    }
}

template <class Real, int DIM, int KERNEL, int T>
cudaError_t launch_fused_t(const FusedLaunch& F, int grid, cudaStream_t st) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(FUSED_THREADS);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_step_fused<Real, DIM, KERNEL, T>, F);
}

template <class Real, int DIM, int KERNEL, int T>
int fused_bps_t() {
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_step_fused<Real, DIM, KERNEL, T>,
                                                  FUSED_THREADS, 0);
    return b;
}

// Launch and blocks per SM of the persistent kernel for one precision and tile shape,
// dispatched on (dim, kernel); each (precision, shape) is its own translation unit.
template <class Real, int T>
cudaError_t fused_launch(const FusedLaunch& F, int grid, cudaStream_t st) {
    const int sel = (F.L.dim == 3 ? 3 : 0) + F.L.kernel;
    switch (sel) {
        case 0: return launch_fused_t<Real, 2, QUINTIC, T>(F, grid, st);
        case 1: return launch_fused_t<Real, 2, WENDLAND_C2, T>(F, grid, st);
        case 2: return launch_fused_t<Real, 2, CUBIC_SPLINE, T>(F, grid, st);
        case 3: return launch_fused_t<Real, 3, QUINTIC, T>(F, grid, st);
        case 4: return launch_fused_t<Real, 3, WENDLAND_C2, T>(F, grid, st);
        default: return launch_fused_t<Real, 3, CUBIC_SPLINE, T>(F, grid, st);
    }
}

template <class Real, int T>
int fused_bps(int dim, int kernel) {
    const int sel = (dim == 3 ? 3 : 0) + kernel;
    switch (sel) {
        case 0: return fused_bps_t<Real, 2, QUINTIC, T>();
        case 1: return fused_bps_t<Real, 2, WENDLAND_C2, T>();
        case 2: return fused_bps_t<Real, 2, CUBIC_SPLINE, T>();
        case 3: return fused_bps_t<Real, 3, QUINTIC, T>();
        case 4: return fused_bps_t<Real, 3, WENDLAND_C2, T>();
        default: return fused_bps_t<Real, 3, CUBIC_SPLINE, T>();
    }
}

}  // namespace sph
