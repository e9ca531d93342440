// Persistent step kernel with float pair arithmetic and 8 lanes per destination.
#include "fused_impl.cuh"

namespace sph {

template cudaError_t fused_launch<float, 8>(const FusedLaunch&, int, cudaStream_t);
template int fused_bps<float, 8>(int, int);

}  // namespace sph
