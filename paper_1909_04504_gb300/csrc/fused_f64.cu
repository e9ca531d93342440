// FP64 instantiations of the persistent step kernel, and the precision dispatch.
#include "fused_impl.cuh"

namespace sph {

cudaError_t launch_fused_f32(const FusedLaunch& F, int T, int grid, cudaStream_t st);
int fused_bps_f32(int dim, int kernel, int T);

cudaError_t launch_fused(const FusedLaunch& F, int T, int grid, cudaStream_t st) {
    if (F.L.precision) return launch_fused_f32(F, T, grid, st);
    return FusedDispatch<double>::launch(F, T, grid, st);
}

int fused_max_blocks_per_sm(int precision, int dim, int kernel, int T) {
    return precision ? fused_bps_f32(dim, kernel, T) : FusedDispatch<double>::bps(dim, kernel, T);
}

}  // namespace sph
