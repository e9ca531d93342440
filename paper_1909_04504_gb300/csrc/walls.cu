// Solid-wall pressure of Adami, Hu and Adams (2012), the wall boundary condition listed
// among the schemes of Sec. 2.3 (scheme option SPH_WALL_ADAMI). Runs between the density
// pass and the momentum pass of an evaluation: each wall particle w takes
//   p_w = (sum_f p_f W_wf + g . sum_f rho_f (x_w - x_f) W_wf) / sum_f W_wf
// over its fluid neighbours f (static walls: no wall acceleration) and the density the
// Tait EOS (Eq. eos) maps to it, rho_w = rho0 (1 + p_w / B)^(1/gamma); a wall with no
// fluid neighbour takes p_w = 0 and rho_w = rho0. The neighbours are those of the
// density pass's list (in continuity mode a wall lists its fluid neighbours only; in
// summation mode every neighbour, the walls among them skipped here). Fluid pressures
// come from the pair-loop shadow, p_f = (p/rho^2)_f rho_f^2; the sums are compensated in
// the pair-loop precision (8 lanes per wall particle, combined by a fixed shuffle tree),
// the quotient and the EOS inversion run in FP64.
#include "pairs_impl.cuh"

namespace sph {

constexpr int WALL_LANES = 8;  // lanes per particle: a wall's list is split among them

// The FP64 pipe of this part runs at 1/64 of FP32, and a warp pays for every FP64
// instruction whatever its active lanes: the reciprocal and the EOS root start from the
// FP32 hardware value and take one Newton step in FP64 (the FP32 start is good to a few
// 2^-23, so one step leaves an error of order 2^-46, far below the sums' rounding).
// The FP32 start needs x and 1/x inside FP32's normal range (the approximation flushes
// subnormals to zero): outside it, and for 0, infinities and NaN, the FP64 divide. A wall
// whose only fluid neighbour sits at the edge of the support has a kernel-weight sum far
// below FP32's range in FP64 mode (1 - q/2 ~ 1e-12 gives ~1e-45).
__device__ __forceinline__ double rcp_fp64(double x) {
    const double ax = fabs(x);
    if (!(ax >= 0x1p-125 && ax <= 0x1p125)) return 1.0 / x;
    const double r = (double)PairMath<float>::rcp((float)x);
    return r * fma(-x, r, 2.0);
}

// x^(1/gamma): for gamma = 7 Newton's step on y^7 = x from the FP32 root; else, or where
// the FP32 root would leave FP32's normal range, pow.
__device__ __forceinline__ double eos_root(double x, const StepConst& C) {
    if (!C.gamma7 || !(x >= 0x1p-120 && x <= 0x1p120)) return pow(x, 1.0 / C.gamma);
    double y = (double)powf((float)x, 1.0f / 7.0f);
    const double y3 = y * y * y;
    const double y6 = y3 * y3;
    y -= fma(y6, y, -x) * (1.0 / 7.0) * rcp_fp64(y6);
    return y;
}

template <class Real, int DIM, int KERNEL>
__global__ void __launch_bounds__(PAIR_THREADS)
k_wall_pressure(const typename V4<Real>::T* __restrict__ P, typename V4<Real>::T* __restrict__ Q,
                Real* __restrict__ R, const uint32_t* __restrict__ skeys, int n,
                const Inst<Real>* __restrict__ tab, const uint32_t* __restrict__ cell_bounds,
                int ninst, ParticleSet S, const uint32_t* __restrict__ nl,
                const uint32_t* __restrict__ cnt, const Control* ctl) {
    if (ctl->status) return;
    constexpr int T = WALL_LANES;
    const Group<T> g;
    const int groups = gridDim.x * (PAIR_THREADS / T);
    for (int i = blockIdx.x * (PAIR_THREADS / T) + (int)threadIdx.x / T; i < n; i += groups) {
        const typename V4<Real>::T pi = P[i];
        if (pi.w > Real(0)) continue;  // fluid (uniform over the group)
        const Inst<Real>& I = tab[find_instance(cell_bounds, ninst, skeys[i])];
        if (!(I.K.flags & F_WALLP)) continue;
        const Real gx = (Real)I.C.g[0], gy = (Real)I.C.g[1], gz = (Real)I.C.g[2];
        Acc<Real> sw, sp, sg;
        sw.zero();
        sp.zero();
        sg.zero();
        const uint32_t k = cnt[i];
        for (uint32_t kk = g.t; kk < k; kk += T) {
            const uint32_t j = nl[(size_t)kk * n + i];
            const typename V4<Real>::T pj = P[j];
            if (!(pj.w > Real(0))) continue;  // wall source
            Real dx, dy, dz;
            const Real r2 = separation<Real, DIM>(pi, pj, I.G, I.K, dx, dy, dz);
            const Real W = I.K.wfac * kernel_w<Real, KERNEL>(PairMath<Real>::sqrt(r2) * I.K.inv_h);
            const Real rho_j = Q[j].w;
            const Real gr = gx * dx + gy * dy + (DIM == 3 ? gz * dz : Real(0));
            sw.add(W);
            sp.add(R[j] * rho_j * rho_j * W);
            sg.add(rho_j * gr * W);
        }
        group_reduce<Real, T>(sw, g);
        group_reduce<Real, T>(sp, g);
        group_reduce<Real, T>(sg, g);
        if (g.t == 0) {
            const double w = sw.value();
            double pw = 0.0, rw = I.C.rho0;
            if (w > 0.0) {
                pw = (sp.value() + sg.value()) * rcp_fp64(w);
                rw = I.C.rho0 * eos_root(1.0 + pw * (1.0 / I.C.B), I.C);
            }
            S.rho[i] = rw;
            reinterpret_cast<Real*>(&Q[i])[3] = (Real)rw;
            R[i] = (Real)(pw * rcp_fp64(rw * rw));
        }
    }
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
