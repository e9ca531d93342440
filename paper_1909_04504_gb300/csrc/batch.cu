// Per-instance reduction of a batched step. A batch holds many independent problems
// (instances) of uneven size in one set of arrays; the sort key is the instance's first
// global cell id plus the local cell id, so a stable sort keeps every instance contiguous
// and, inside it, in the order a single run of that instance would have. The step kernels
// are the single-problem kernels (they read every constant from the instance table), so
// an instance of a batch computes bitwise what its single run computes.
#include "sph_device.cuh"
#include "sph_launch.h"
#include "reduce_impl.cuh"

namespace sph {

// One block per instance over its contiguous cell-order segment.
template <class Real>
__global__ void __launch_bounds__(256)
k_batch_reduce(ParticleSet S, const uint32_t* __restrict__ pcount, const uint32_t* __restrict__ off,
               const Inst<Real>* __restrict__ tab, int ninst, int dim, double* __restrict__ idt,
               double* __restrict__ it, double* __restrict__ irec, int kick, Control* ctl) {
    __shared__ double red[8][10];
    if (ctl->status) return;
    const int inst = blockIdx.x;
    if (inst >= ninst) return;
    batch_reduce_inst<Real, 256>(S, pcount, off, tab[inst], inst, dim, idt, it, irec, kick, ctl, red);
}

// ---------------------------------------------------------------- launchers
void launch_batch_reduce(const StepLaunch& L, cudaStream_t st) {
    if (L.precision)
        k_batch_reduce<float><<<L.ninst, 256, 0, st>>>(L.S, L.pcount, L.off, (const Inst<float>*)L.tab,
                                                       L.ninst, L.dim, L.idt, L.it, L.irec, L.kick,
                                                       L.ctl);
    else
        k_batch_reduce<double><<<L.ninst, 256, 0, st>>>(L.S, L.pcount, L.off,
                                                        (const Inst<double>*)L.tab, L.ninst, L.dim,
                                                        L.idt, L.it, L.irec, L.kick, L.ctl);
}

}  // namespace sph
