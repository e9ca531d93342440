// Dispatch of one right-hand-side evaluation (density pass, then momentum pass) to the
// kernel instantiation of the context's precision and group size (the instantiations, per
// precision and group size, are pairs_f32_t1.cu ... pairs_f64_t8.cu; they dispatch on the
// dimension and smoothing kernel). The kernels themselves are in pairs_impl.cuh.
#include "sph_device.cuh"
#include "sph_launch.h"
#include "pair_units.h"

namespace sph {

template <class Real>
static int pairs_bps_p(int pass, int dim, int kernel, int T, int single) {
    switch (T) {
        case 1: return pair_bps<Real, 1>(pass, dim, kernel, single);
        case 2: return pair_bps<Real, 2>(pass, dim, kernel, single);
        case 4: return pair_bps<Real, 4>(pass, dim, kernel, single);
        default: return pair_bps<Real, 8>(pass, dim, kernel, single);
    }
}

template <class Real>
static void density_p(const StepLaunch& L, cudaStream_t st) {
    switch (L.group_d) {
        case 1: pair_density<Real, 1>(L, st); break;
        case 2: pair_density<Real, 2>(L, st); break;
        case 4: pair_density<Real, 4>(L, st); break;
        default: pair_density<Real, 8>(L, st); break;
    }
}

template <class Real>
static void momentum_p(const StepLaunch& L, cudaStream_t st) {
    switch (L.group_m) {
        case 1: pair_momentum<Real, 1>(L, st); break;
        case 2: pair_momentum<Real, 2>(L, st); break;
        case 4: pair_momentum<Real, 4>(L, st); break;
        default: pair_momentum<Real, 8>(L, st); break;
    }
}

int pair_threads() { return 128; }

void launch_density_pass(const StepLaunch& L, cudaStream_t st) {
    if (L.precision) density_p<float>(L, st);
    else density_p<double>(L, st);
}

void launch_momentum_pass(const StepLaunch& L, cudaStream_t st) {
    if (L.precision) momentum_p<float>(L, st);
    else momentum_p<double>(L, st);
}

void launch_pairs(const StepLaunch& L, cudaStream_t st) {
    launch_density_pass(L, st);
    launch_momentum_pass(L, st);
    if (!L.finalize) launch_batch_reduce(L, st);
}

int pairs_max_blocks_per_sm(int precision, int pass, int dim, int kernel, int T, int single) {
    return precision ? pairs_bps_p<float>(pass, dim, kernel, T, single)
                     : pairs_bps_p<double>(pass, dim, kernel, T, single);
}

}  // namespace sph
