// Entry points of the persistent-step instantiations, one translation unit per pair-loop
// precision and tile shape (T lanes per destination) so that they compile in parallel.
#pragma once

#include "sph_launch.h"

namespace sph {

template <class Real, int T>
cudaError_t fused_launch(const FusedLaunch& F, int grid, cudaStream_t st);
template <class Real, int T>
int fused_bps(int dim, int kernel);

}  // namespace sph
