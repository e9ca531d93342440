// Persistent step kernel with double pair arithmetic and 8 lanes per destination.
#include "fused_impl.cuh"

namespace sph {

template cudaError_t fused_launch<double, 8>(const FusedLaunch&, int, cudaStream_t);
template int fused_bps<double, 8>(int, int);

}  // namespace sph
