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
    batch_chunk_partials<Real, 256>(S, pcount, off, tab[blockIdx.y], blockIdx.y, blockIdx.x, dim, part,
                                    red);
}

template <class Real>
__global__ void __launch_bounds__(256)
k_batch_finish(const Inst<Real>* __restrict__ tab, int ninst, const double* __restrict__ part,
               double* __restrict__ idt, double* __restrict__ it, double* __restrict__ irec, int kick,
               Control* ctl) {
    if (ctl->status) return;
    const int inst = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (inst >= ninst) return;
    batch_finish_warp<Real>(tab[inst], inst, part, idt, it, irec, kick, ctl);
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
