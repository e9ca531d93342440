// Persistent step kernel with float pair arithmetic and 4 lanes per destination.
#include "fused_impl.cuh"

namespace sph {

template cudaError_t fused_launch<float, 4>(const FusedLaunch&, int, cudaStream_t);
template int fused_bps<float, 4>(int, int);

}  // namespace sph
