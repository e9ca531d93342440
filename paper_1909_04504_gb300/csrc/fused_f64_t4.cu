// Persistent step kernel with double pair arithmetic and 4 lanes per destination.
#include "fused_impl.cuh"

namespace sph {

template cudaError_t fused_launch<double, 4>(const FusedLaunch&, int, cudaStream_t);
template int fused_bps<double, 4>(int, int);

}  // namespace sph
