// Dispatch of the persistent step kernel on the pair-loop precision and the tile shape;
// the instantiations are in fused_f32_t1.cu ... fused_f64_t8.cu.
#include "fused_units.h"

namespace sph {

template <class Real>
static cudaError_t fused_launch_p(const FusedLaunch& F, int T, int grid, cudaStream_t st) {
    switch (T) {
        case 1: return fused_launch<Real, 1>(F, grid, st);
        case 2: return fused_launch<Real, 2>(F, grid, st);
        case 4: return fused_launch<Real, 4>(F, grid, st);
        default: return fused_launch<Real, 8>(F, grid, st);
    }
}

template <class Real>
static int fused_bps_p(int dim, int kernel, int T) {
    switch (T) {
        case 1: return fused_bps<Real, 1>(dim, kernel);
        case 2: return fused_bps<Real, 2>(dim, kernel);
        case 4: return fused_bps<Real, 4>(dim, kernel);
        default: return fused_bps<Real, 8>(dim, kernel);
    }
}

cudaError_t launch_fused(const FusedLaunch& F, int T, int grid, cudaStream_t st) {
    return F.L.precision ? fused_launch_p<float>(F, T, grid, st) : fused_launch_p<double>(F, T, grid, st);
}

int fused_max_blocks_per_sm(int precision, int dim, int kernel, int T) {
    return precision ? fused_bps_p<float>(dim, kernel, T) : fused_bps_p<double>(dim, kernel, T);
}

}  // namespace sph
