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
#pragma once

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

// Wall particles i = block * (NTH / WALL_LANES) + group, with a stride of nblocks blocks:
// the per-wall body shared by the wall kernel and the persistent step.
template <class Real, int DIM, int KERNEL, int NTH>
__device__ __forceinline__ void wall_pressure_range(int block, int nblocks,
                                                    const typename V4<Real>::T* __restrict__ P,
                                                    typename V4<Real>::T* __restrict__ Q,
                                                    Real* __restrict__ R,
                                                    const uint32_t* __restrict__ skeys, int n,
                                                    const Inst<Real>* __restrict__ tab,
                                                    const uint32_t* __restrict__ cell_bounds,
                                                    int ninst, const ParticleSet& S,
                                                    const uint32_t* __restrict__ nl,
                                                    const uint32_t* __restrict__ cnt) {
    constexpr int T = WALL_LANES;
    const Group<T> g;
    const int groups = nblocks * (NTH / T);
    for (int i = block * (NTH / T) + (int)threadIdx.x / T; i < n; i += groups) {
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

}  // namespace sph
