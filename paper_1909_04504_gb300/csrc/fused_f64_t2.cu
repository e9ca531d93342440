// Persistent step kernel with double pair arithmetic and 2 lanes per destination.
#include "fused_impl.cuh"

namespace sph {

template cudaError_t fused_launch<double, 2>(const FusedLaunch&, int, cudaStream_t);
template int fused_bps<double, 2>(int, int);

}  // namespace sph
