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
    const bool fluid = !(S.tag[i] & WALL_BIT);
    int c[3] = {0, 0, 0};
    for (int d = 0; d < G.dim; ++d) {
        double x = S.x[d][i];
        if (drift && fluid) {
            double uh = S.u[d][i] + 0.5 * dt * S.a[d][i];
            x = x + dt * (uh + S.xs[d][i]);
            if (G.periodic[d] && !(x >= G.lo[d] && x < G.hi[d])) {
                double k = floor(__ddiv_rn(__dsub_rn(x, G.lo[d]), G.L[d]));
                x = __dsub_rn(x, __dmul_rn(k, G.L[d]));
                if (x >= G.hi[d]) x = __dsub_rn(x, G.L[d]);
                if (x < G.lo[d]) x = G.lo[d];
            }
            S.x[d][i] = x;
        }
        const float xf = __double2float_rn(x);
        const double xm = C.precision ? (double)xf : x;
        c[d] = cell_coord_screened(xm, xf, G.lo[d], G.cs[d], G.lo_f[d], G.inv_cs_f[d], G.nc[d],
                                   &clamped);
    }
    return (uint32_t)(c[0] + G.nc[0] * (c[1] + G.nc[1] * c[2]));
}

// Gather of particle o (previous order) into position k of the cell order. kick: the
// predictor half-kick of the fluid velocity (the density is advanced later, like the
// positions, by the density pass). Rates are carried along only outside a step
// (carry_rates). Writes the pair-loop shadow P = (x, y, z, +-m) with the sign marking
// walls and Q = (u, v, w, .); the density pass that follows writes Q.w = rho and p / rho^2.
template <class Real>
__device__ __forceinline__ void reorder_one(const ParticleSet& in, const ParticleSet& out, int k,
                                            int o, int dim, double dt, int kick, int carry_rates,
                                            typename V4<Real>::T* __restrict__ P,
                                            typename V4<Real>::T* __restrict__ Q) {
    const uint32_t tag = in.tag[o];
    const bool fluid = !(tag & WALL_BIT);
    double x[3] = {0, 0, 0}, u[3] = {0, 0, 0};
    for (int d = 0; d < dim; ++d) {
        x[d] = in.x[d][o];
        u[d] = in.u[d][o];
        if (kick && fluid) u[d] += 0.5 * dt * in.a[d][o];
        out.x[d][k] = x[d];
        out.u[d][k] = u[d];
    }
    const double rho = in.rho[o];
    const double m = in.m[o];
    out.rho[k] = rho;
    out.m[k] = m;
    out.tag[k] = tag;
    if (carry_rates) {
        out.arho[k] = in.arho[o];
        for (int d = 0; d < dim; ++d) {
            out.a[d][k] = in.a[d][o];
            out.xs[d][k] = in.xs[d][o];
        }
    }
    typename V4<Real>::T pv, qv;
    pv.x = (Real)x[0]; pv.y = (Real)x[1]; pv.z = (Real)x[2];
    pv.w = (Real)(fluid ? m : -m);
    qv.x = (Real)u[0]; qv.y = (Real)u[1]; qv.z = (Real)u[2];
    qv.w = Real(0);  // the density pass writes it
    P[k] = pv;
    Q[k] = qv;
}

}  // namespace sph
