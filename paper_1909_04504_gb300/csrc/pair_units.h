// Entry points of the pair-pass instantiations, one translation unit per pair-loop
// precision and tile shape (T lanes per destination) so that they compile in parallel:
// blocks per SM of a pass, and the density and momentum launches.
#pragma once

#include "sph_launch.h"

namespace sph {

template <class Real, int T>
int pair_bps(int pass, int dim, int kernel, int single);
template <class Real, int T>
void pair_density(const StepLaunch& L, cudaStream_t st);
template <class Real, int T>
void pair_momentum(const StepLaunch& L, cudaStream_t st);

}  // namespace sph
