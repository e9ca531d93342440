// Instantiations of the pair-loop kernels for float pair arithmetic (one translation unit
// per precision so that the two compile in parallel).
#include "pairs_impl.cuh"

namespace sph {

int pairs_bps_f32(int pass, int dim, int kernel, int T) {
    switch (T) {
        case 1: return PairDispatch<float>::bps_t<1>(pass, dim, kernel);
        case 2: return PairDispatch<float>::bps_t<2>(pass, dim, kernel);
        case 4: return PairDispatch<float>::bps_t<4>(pass, dim, kernel);
        default: return PairDispatch<float>::bps_t<8>(pass, dim, kernel);
    }
}

void launch_density_f32(const StepLaunch& L, cudaStream_t st) {
    switch (L.group_d) {
        case 1: PairDispatch<float>::density_t<1>(L, st); break;
        case 2: PairDispatch<float>::density_t<2>(L, st); break;
        case 4: PairDispatch<float>::density_t<4>(L, st); break;
        default: PairDispatch<float>::density_t<8>(L, st); break;
    }
}

void launch_momentum_f32(const StepLaunch& L, cudaStream_t st) {
    switch (L.group_m) {
        case 1: PairDispatch<float>::momentum_t<1>(L, st); break;
        case 2: PairDispatch<float>::momentum_t<2>(L, st); break;
        case 4: PairDispatch<float>::momentum_t<4>(L, st); break;
        default: PairDispatch<float>::momentum_t<8>(L, st); break;
    }
}

}  // namespace sph
