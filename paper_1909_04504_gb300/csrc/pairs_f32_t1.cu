// Pair-loop kernels with float pair arithmetic and 1 lane per destination.
#include "pairs_impl.cuh"

namespace sph {

template int pair_bps<float, 1>(int, int, int, int);
template void pair_density<float, 1>(const StepLaunch&, cudaStream_t);
template void pair_momentum<float, 1>(const StepLaunch&, cudaStream_t);

}  // namespace sph
