// Pair-loop kernels with double pair arithmetic and 4 lanes per destination.
#include "pairs_impl.cuh"

namespace sph {

template int pair_bps<double, 4>(int, int, int, int);
template void pair_density<double, 4>(const StepLaunch&, cudaStream_t);
template void pair_momentum<double, 4>(const StepLaunch&, cudaStream_t);

}  // namespace sph
