// Per-particle bodies of the neighbour-build stages, shared by the single-problem
// kernels (nnps.cu) and the batched ones (batch.cu).
#pragma once

#include "sph_device.cuh"

namespace sph {

// Largest k in [0, count) with bounds[k] <= v (bounds ascending, bounds[0] = 0): the
// instance of a particle (by original id) or of a cell (by global cell id).
__device__ __forceinline__ int find_instance(const uint32_t* __restrict__ bounds, int count, uint32_t v) {
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (bounds[mid] <= v) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Drift + cell key of particle i in the current order (Sec. 2.1 drift, Sec. 2.2 binning):
// for fluid, u_half = u + dt/2 a and x <- wrap(x + dt (u_half + xsph)), written back in
// place; then the linear cell id of the position rounded to the pair-loop precision.
__device__ __forceinline__ uint32_t drift_key_one(const ParticleSet& S, int i, const Grid& G,
                                                  const StepConst& C, double dt, int drift,
                                                  int& clamped) {
    // every load before any store: the compiler cannot tell that the stores to x do not
    // alias the other arrays, and interleaving them would serialise the round trips
    const int dim = G.dim;
    const bool fluid = !(S.tag[i] & WALL_BIT);
    double x[3] = {0, 0, 0};
#pragma unroll
    for (int d = 0; d < 3; ++d)
        if (d < dim) x[d] = S.x[d][i];
    if (drift && fluid) {
        double u[3] = {0, 0, 0}, a[3] = {0, 0, 0}, xs[3] = {0, 0, 0};
#pragma unroll
        for (int d = 0; d < 3; ++d)
            if (d < dim) {
                u[d] = S.u[d][i];
                a[d] = S.a[d][i];
                xs[d] = S.xs[d][i];
            }
#pragma unroll
        for (int d = 0; d < 3; ++d)
            if (d < dim) {
                const double uh = fma_rn(0.5 * dt, a[d], u[d]);
                double xn = fma_rn(dt, uh + xs[d], x[d]);
                if (G.periodic[d] && !(xn >= G.lo[d] && xn < G.hi[d])) {
                    const double k = floor(__ddiv_rn(__dsub_rn(xn, G.lo[d]), G.L[d]));
                    xn = __dsub_rn(xn, __dmul_rn(k, G.L[d]));
                    if (xn >= G.hi[d]) xn = __dsub_rn(xn, G.L[d]);
                    if (xn < G.lo[d]) xn = G.lo[d];
                }
                x[d] = xn;
            }
#pragma unroll
        for (int d = 0; d < 3; ++d)
            if (d < dim) S.x[d][i] = x[d];
    }
    int c[3] = {0, 0, 0};
#pragma unroll
    for (int d = 0; d < 3; ++d)
        if (d < dim) {
            c[d] = cell_coord_screened(x[d], __double2float_rn(x[d]), C.precision, G.lo[d],
                                       G.cs[d], G.lo_f[d], G.inv_cs_f[d], G.nc[d], &clamped);
        }
    return (uint32_t)(c[0] + G.nc[0] * (c[1] + G.nc[1] * c[2]));
}

// Gather of particle o (previous order) into position k of the cell order. kick: the
// predictor half-kick of the fluid velocity (the density is advanced later, like the
// positions, by the density pass). Rates are carried along only outside a step
// (carry_rates). Writes the pair-loop shadow P = (x, y, z, +-m) with the sign marking
// walls and Q = (u, v, w, .); the density pass that follows writes Q.w = rho and p / rho^2.
// edac: the pressure p (a state variable of the EDAC form) is gathered too and its value
// at the start of the evaluation goes to Q.w, which the density pass then only reads.
// E (FP32 pair loops, may be null): the residuals x - (float)x, y - (float)y, z - (float)z
// of the rounded positions (each exact in FP64, then rounded), so that the pair sums form
// separations as (x_i - x_j) + (e_i - e_j) to nearly FP32 precision of the separation
// itself, where x_i - x_j alone carries the rounding of positions far larger than it.
template <class Real>
__device__ __forceinline__ void reorder_one(const ParticleSet& in, const ParticleSet& out, int k,
                                            int o, int dim, double dt, int kick, int carry_rates,
                                            typename V4<Real>::T* __restrict__ P,
                                            typename V4<Real>::T* __restrict__ Q,
                                            F4* __restrict__ E = nullptr, int edac = 0) {
    // every load of particle o before any store (the output arrays could alias the inputs
    // as far as the compiler knows); the acceleration is read for walls too (it is zero
    // there) so that no load waits for the tag
    const uint32_t tag = in.tag[o];
    double x[3] = {0, 0, 0}, u[3] = {0, 0, 0}, a[3] = {0, 0, 0}, xs[3] = {0, 0, 0};
#pragma unroll
    for (int d = 0; d < 3; ++d)
        if (d < dim) {
            x[d] = in.x[d][o];
            u[d] = in.u[d][o];
            if (kick || carry_rates) a[d] = in.a[d][o];
            if (carry_rates) xs[d] = in.xs[d][o];
        }
    const double rho = in.rho[o];
    const double m = in.m[o];
    const double pe = edac ? in.p[o] : 0.0;
    const double arho = carry_rates ? in.arho[o] : 0.0;
    const bool fluid = !(tag & WALL_BIT);
    double uk[3] = {u[0], u[1], u[2]};
    if (kick && fluid)
#pragma unroll
        for (int d = 0; d < 3; ++d)
            if (d < dim) uk[d] = fma_rn(0.5 * dt, a[d], uk[d]);
#pragma unroll
    for (int d = 0; d < 3; ++d)
        if (d < dim) {
            out.x[d][k] = x[d];
            out.u[d][k] = uk[d];
        }
    out.rho[k] = rho;
    out.m[k] = m;
    if (edac) out.p[k] = pe;
    out.tag[k] = tag;
    if (carry_rates) {
        out.arho[k] = arho;
#pragma unroll
        for (int d = 0; d < 3; ++d)
            if (d < dim) {
                out.a[d][k] = a[d];
                out.xs[d][k] = xs[d];
            }
    }
    typename V4<Real>::T pv, qv;
    pv.x = (Real)x[0]; pv.y = (Real)x[1]; pv.z = (Real)x[2];
    pv.w = (Real)(fluid ? m : -m);
    qv.x = (Real)uk[0]; qv.y = (Real)uk[1]; qv.z = (Real)uk[2];
    qv.w = edac ? (Real)pe : Real(0);  // the density pass writes rho; EDAC: the pressure p^n
    P[k] = pv;
    Q[k] = qv;
    if (E) {
        F4 ev;
        ev.x = (float)(x[0] - (double)(float)x[0]);
        ev.y = (float)(x[1] - (double)(float)x[1]);
        ev.z = (float)(x[2] - (double)(float)x[2]);
        ev.w = 0.0f;
        E[k] = ev;
    }
}

}  // namespace sph
