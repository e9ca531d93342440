// Pair-loop kernels with double pair arithmetic and 1 lane per destination.
#include "pairs_impl.cuh"

namespace sph {

template int pair_bps<double, 1>(int, int, int, int);
template void pair_density<double, 1>(const StepLaunch&, cudaStream_t);
template void pair_momentum<double, 1>(const StepLaunch&, cudaStream_t);

}  // namespace sph
