// Instantiations of the pair-loop kernels for double pair arithmetic (one translation unit
// per precision so that the two compile in parallel).
#include "pairs_impl.cuh"

namespace sph {

int pairs_bps_f64(int pass, int dim, int kernel, int T) {
    switch (T) {
        case 1: return PairDispatch<double>::bps_t<1>(pass, dim, kernel);
        case 2: return PairDispatch<double>::bps_t<2>(pass, dim, kernel);
        case 4: return PairDispatch<double>::bps_t<4>(pass, dim, kernel);
        default: return PairDispatch<double>::bps_t<8>(pass, dim, kernel);
    }
}

void launch_density_f64(const StepLaunch& L, cudaStream_t st) {
    switch (L.group_d) {
        case 1: PairDispatch<double>::density_t<1>(L, st); break;
        case 2: PairDispatch<double>::density_t<2>(L, st); break;
        case 4: PairDispatch<double>::density_t<4>(L, st); break;
        default: PairDispatch<double>::density_t<8>(L, st); break;
    }
}

void launch_momentum_f64(const StepLaunch& L, cudaStream_t st) {
    switch (L.group_m) {
        case 1: PairDispatch<double>::momentum_t<1>(L, st); break;
        case 2: PairDispatch<double>::momentum_t<2>(L, st); break;
        case 4: PairDispatch<double>::momentum_t<4>(L, st); break;
        default: PairDispatch<double>::momentum_t<8>(L, st); break;
    }
}

}  // namespace sph
