// Persistent step kernel with double pair arithmetic and 1 lane per destination.
#include "fused_impl.cuh"

namespace sph {

template cudaError_t fused_launch<double, 1>(const FusedLaunch&, int, cudaStream_t);
template int fused_bps<double, 1>(int, int);

}  // namespace sph
