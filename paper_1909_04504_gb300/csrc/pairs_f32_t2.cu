// Pair-loop kernels with float pair arithmetic and 2 lanes per destination.
#include "pairs_impl.cuh"

namespace sph {

template int pair_bps<float, 2>(int, int, int, int);
template void pair_density<float, 2>(const StepLaunch&, cudaStream_t);
template void pair_momentum<float, 2>(const StepLaunch&, cudaStream_t);

}  // namespace sph
