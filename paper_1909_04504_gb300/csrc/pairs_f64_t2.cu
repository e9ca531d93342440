// Pair-loop kernels with double pair arithmetic and 2 lanes per destination.
#include "pairs_impl.cuh"

namespace sph {

template int pair_bps<double, 2>(int, int, int, int);
template void pair_density<double, 2>(const StepLaunch&, cudaStream_t);
template void pair_momentum<double, 2>(const StepLaunch&, cudaStream_t);

}  // namespace sph
