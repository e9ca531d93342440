// Solid-wall pressure pass (the body and its reading: walls_impl.cuh).
#include "walls_impl.cuh"

namespace sph {

template <class Real, int DIM, int KERNEL>
__global__ void __launch_bounds__(PAIR_THREADS)
k_wall_pressure(const typename V4<Real>::T* __restrict__ P, typename V4<Real>::T* __restrict__ Q,
                Real* __restrict__ R, const uint32_t* __restrict__ skeys, int n,
                const Inst<Real>* __restrict__ tab, const uint32_t* __restrict__ cell_bounds,
                int ninst, ParticleSet S, const uint32_t* __restrict__ nl,
                const uint32_t* __restrict__ cnt, const Control* ctl) {
    if (ctl->status) return;
    wall_pressure_range<Real, DIM, KERNEL, PAIR_THREADS>(blockIdx.x, gridDim.x, P, Q, R, skeys, n, tab,
                                                         cell_bounds, ninst, S, nl, cnt);
}

template <class Real, int DIM, int KERNEL>
static void wall_pressure_t(const StepLaunch& L, cudaStream_t st) {
    using V = typename V4<Real>::T;
    long long want = ((long long)L.n * WALL_LANES + PAIR_THREADS - 1) / PAIR_THREADS;
    const long long cap = (long long)L.sms * 16;
    const int g = (int)(want < 1 ? 1 : (want > cap ? cap : want));
    k_wall_pressure<Real, DIM, KERNEL><<<g, PAIR_THREADS, 0, st>>>(
        (const V*)L.P, (V*)L.Q, (Real*)L.R, L.skeys, L.n, (const Inst<Real>*)L.tab, L.cell_bounds,
        L.ninst, L.S, L.nl, L.cnt, L.ctl);
}

void launch_wall_pressure(const StepLaunch& L, cudaStream_t st) {
    const int sel = (L.precision ? 6 : 0) + (L.dim == 3 ? 3 : 0) + L.kernel;
    switch (sel) {
        case 0: wall_pressure_t<double, 2, QUINTIC>(L, st); break;
        case 1: wall_pressure_t<double, 2, WENDLAND_C2>(L, st); break;
        case 2: wall_pressure_t<double, 2, CUBIC_SPLINE>(L, st); break;
        case 3: wall_pressure_t<double, 3, QUINTIC>(L, st); break;
        case 4: wall_pressure_t<double, 3, WENDLAND_C2>(L, st); break;
        case 5: wall_pressure_t<double, 3, CUBIC_SPLINE>(L, st); break;
        case 6: wall_pressure_t<float, 2, QUINTIC>(L, st); break;
        case 7: wall_pressure_t<float, 2, WENDLAND_C2>(L, st); break;
        case 8: wall_pressure_t<float, 2, CUBIC_SPLINE>(L, st); break;
        case 9: wall_pressure_t<float, 3, QUINTIC>(L, st); break;
        case 10: wall_pressure_t<float, 3, WENDLAND_C2>(L, st); break;
        default: wall_pressure_t<float, 3, CUBIC_SPLINE>(L, st); break;
    }
}

}  // namespace sph
