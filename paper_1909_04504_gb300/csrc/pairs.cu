// Dispatch of one right-hand-side evaluation (density pass, then momentum pass) to the
// kernel instantiation of the context's precision, dimension, smoothing kernel and group
// size. The kernels themselves are in pairs_impl.cuh.
#include "sph_device.cuh"
#include "sph_launch.h"

namespace sph {

int pairs_bps_f32(int pass, int dim, int kernel, int T);
int pairs_bps_f64(int pass, int dim, int kernel, int T);
void launch_density_f32(const StepLaunch& L, cudaStream_t st);
void launch_density_f64(const StepLaunch& L, cudaStream_t st);
void launch_momentum_f32(const StepLaunch& L, cudaStream_t st);
void launch_momentum_f64(const StepLaunch& L, cudaStream_t st);

int pair_threads() { return 128; }

void launch_density_pass(const StepLaunch& L, cudaStream_t st) {
    if (L.precision) launch_density_f32(L, st);
    else launch_density_f64(L, st);
}

void launch_momentum_pass(const StepLaunch& L, cudaStream_t st) {
    if (L.precision) launch_momentum_f32(L, st);
    else launch_momentum_f64(L, st);
}

void launch_pairs(const StepLaunch& L, cudaStream_t st) {
    launch_density_pass(L, st);
    launch_momentum_pass(L, st);
    if (!L.finalize) launch_batch_reduce(L, st);
}

int pairs_max_blocks_per_sm(int precision, int pass, int dim, int kernel, int T) {
    return precision ? pairs_bps_f32(pass, dim, kernel, T) : pairs_bps_f64(pass, dim, kernel, T);
}

}  // namespace sph
