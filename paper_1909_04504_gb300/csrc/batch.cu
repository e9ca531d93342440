// Per-instance reduction of a batched step. A batch holds many independent problems
// (instances) of uneven size in one set of arrays; the sort key is the instance's first
// global cell id plus the local cell id, so a stable sort keeps every instance contiguous
// and, inside it, in the order a single run of that instance would have. The step kernels
// are the single-problem kernels (they read every constant from the instance table), so
// an instance of a batch computes bitwise what its single run computes.
#include "sph_device.cuh"
#include "sph_launch.h"
#include "batch_impl.cuh"

namespace sph {

// Two stages, so the reduction spreads over the whole GPU: BATCH_SPLIT blocks per instance
// reduce consecutive chunks of its contiguous cell-order segment into partials, then one
// warp per instance combines its partials in a fixed order and writes the record.
template <class Real>
__global__ void __launch_bounds__(256)
k_batch_partials(ParticleSet S, const uint32_t* __restrict__ pcount, const uint32_t* __restrict__ off,
                 const Inst<Real>* __restrict__ tab, int ninst, int dim, double* __restrict__ part,
                 const Control* ctl) {
    __shared__ double red[8][10];
    if (ctl->status) return;
    const int inst = blockIdx.y, chunk_id = blockIdx.x;
    const uint32_t b0 = off[tab[inst].cell_base], e0 = off[tab[inst].cell_base_end];
    const uint32_t chunk = (e0 - b0 + BATCH_SPLIT - 1) / BATCH_SPLIT;
    const uint32_t b = b0 + chunk_id * chunk;
    const uint32_t e = b + chunk < e0 ? b + chunk : e0;
    double o[10];
    batch_partial<256>(S, pcount, b < e0 ? b : e0, b < e0 ? e : e0, dim, o, red);
    if (threadIdx.x == 0)
        for (int q = 0; q < 10; ++q) part[((size_t)inst * BATCH_SPLIT + chunk_id) * 10 + q] = o[q];
}

template <class Real>
__global__ void __launch_bounds__(256)
k_batch_finish(const Inst<Real>* __restrict__ tab, int ninst, const double* __restrict__ part,
               double* __restrict__ idt, double* __restrict__ it, double* __restrict__ irec, int kick,
               Control* ctl) {
    if (ctl->status) return;
    const int inst = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (inst >= ninst) return;
    double v[10];
    for (int q = 0; q < 10; ++q)
        v[q] = lane < BATCH_SPLIT ? part[((size_t)inst * BATCH_SPLIT + lane) * 10 + q] : 0.0;
    for (int o2 = 16; o2 > 0; o2 >>= 1)
        for (int q = 0; q < 10; ++q) {
            const double y = __shfl_down_sync(0xffffffffu, v[q], o2);
            v[q] = (q >= 4 && q <= 6) ? fmax(v[q], y) : v[q] + y;
        }
    if (lane == 0) batch_finish_inst<Real>(tab[inst], inst, v, idt, it, irec, kick, ctl);
}

// ---------------------------------------------------------------- launchers
template <class Real>
void batch_reduce_t(const StepLaunch& L, cudaStream_t st) {
    const Inst<Real>* tab = (const Inst<Real>*)L.tab;
    k_batch_partials<Real><<<dim3(BATCH_SPLIT, L.ninst), 256, 0, st>>>(L.S, L.pcount, L.off, tab,
                                                                      L.ninst, L.dim, L.bpart, L.ctl);
    const int warps = L.ninst, blocks = (warps * 32 + 255) / 256;
    k_batch_finish<Real><<<blocks, 256, 0, st>>>(tab, L.ninst, L.bpart, L.idt, L.it, L.irec, L.kick,
                                                L.ctl);
}

void launch_batch_reduce(const StepLaunch& L, cudaStream_t st) {
    if (L.precision) batch_reduce_t<float>(L, st);
    else batch_reduce_t<double>(L, st);
}

}  // namespace sph
