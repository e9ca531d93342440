// FP32 pair-loop instantiations of the persistent step kernel.
#include "fused_impl.cuh"

namespace sph {

cudaError_t launch_fused_f32(const FusedLaunch& F, int T, int grid, cudaStream_t st) {
    return FusedDispatch<float>::launch(F, T, grid, st);
}
int fused_bps_f32(int dim, int kernel, int T) { return FusedDispatch<float>::bps(dim, kernel, T); }

}  // namespace sph
