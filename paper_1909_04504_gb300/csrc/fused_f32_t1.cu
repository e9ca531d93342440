// Persistent step kernel with float pair arithmetic and 1 lane per destination.
#include "fused_impl.cuh"

namespace sph {

template cudaError_t fused_launch<float, 1>(const FusedLaunch&, int, cudaStream_t);
template int fused_bps<float, 1>(int, int);

}  // namespace sph
