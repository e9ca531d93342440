// End-of-evaluation bookkeeping (Sec. 2.1 step control): the diagnostics record, the
// history entry, the time, the next dt (fixed, or the CFL-type criteria) and the status,
// for a single problem (from already reduced totals) and per batch instance (a block
// reduction over the instance's contiguous cell-order segment). Shared by the per-phase
// kernels and the persistent step kernel.
#pragma once

#include "sph_device.cuh"
#include "sph_launch.h"

namespace sph {

// Next time step: dt_fixed if positive, else min(0.25 h / (c0 + max|u|),
// 0.25 sqrt(h / max|a|), 0.125 h^2 / nu).
__device__ __forceinline__ double next_dt(const StepConst& C, double umax, double amax) {
    double dn = C.dt_fixed;
    if (!(dn > 0.0)) {
        dn = 0.25 * C.h / (C.c0 + umax);
        if (amax > 0.0) dn = fmin(dn, 0.25 * sqrt(C.h / amax));
        if (C.nu > 0.0) dn = fmin(dn, 0.125 * C.h * C.h / C.nu);
    }
    return dn;
}

// Single problem. out: px py pz ke u2max a2max bad pairs candidates wall-pairs.
__device__ __forceinline__ void finish_single(Control* ctl, double* __restrict__ history,
                                              const StepConst& C, double dt, int kick,
                                              const double* out) {
    double* rec = ctl->rec;
    if (kick) {
        ctl->t += dt;
        ctl->step += 1;
    }
    rec[0] = ctl->t;
    rec[1] = kick ? dt : 0.0;
    rec[2] = out[3];
    rec[3] = sqrt(out[4]);
    rec[4] = out[0];
    rec[5] = out[1];
    rec[6] = out[2];
    rec[7] = sqrt(out[5]);
    rec[8] = out[7];
    rec[9] = out[8];
    rec[10] = (double)ctl->step;
    rec[11] = (double)ctl->outside;
    rec[12] = out[9];
    if (out[6] != 0.0) atomicOr(&ctl->status, ST_NONFINITE);
    ctl->dt = next_dt(C, rec[3], rec[7]);
    if (kick) {
        double* hrec = history + (size_t)(ctl->hist_count % HIST_CAP) * DIAG_N;
        for (int k = 0; k < DIAG_N; ++k) hrec[k] = rec[k];
        ctl->hist_count += 1;
    }
    __threadfence();
}

// FP64 diagnostics of the particles [b, e) of the cell order (one block of NT threads,
// red: NT/32 x 10 doubles of shared memory), in a fixed order; valid in thread 0:
// px py pz ke max|u|^2 max|a|^2 bad pairs candidates wall-pairs.
template <int NT>
__device__ __forceinline__ void batch_partial(const ParticleSet& S,
                                              const uint32_t* __restrict__ pcount, uint32_t b,
                                              uint32_t e, int dim, double* o, double (*red)[10]) {
    double v[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (uint32_t k = b + threadIdx.x; k < e; k += NT) {
        const bool fluid = !(S.tag[k] & WALL_BIT);
        const double np = (double)pcount[2 * (size_t)k], nc = (double)pcount[2 * (size_t)k + 1];
        v[7] += np;
        v[8] += nc;
        if (!fluid) {
            v[9] += np;
            if (!isfinite(S.rho[k])) v[6] = 1.0;
            continue;
        }
        double u2 = 0, a2 = 0;
        for (int d = 0; d < dim; ++d) {
            const double u = S.u[d][k], a = S.a[d][k];
            u2 += u * u;
            a2 += a * a;
            if (d == 0) v[0] += S.m[k] * u;
            if (d == 1) v[1] += S.m[k] * u;
            if (d == 2) v[2] += S.m[k] * u;
            if (!isfinite(u) || !isfinite(S.x[d][k])) v[6] = 1.0;
        }
        if (!isfinite(S.rho[k]) || !isfinite(a2)) v[6] = 1.0;
        v[3] += 0.5 * S.m[k] * u2;
        v[4] = fmax(v[4], u2);
        v[5] = fmax(v[5], a2);
    }
    for (int o2 = 16; o2 > 0; o2 >>= 1)
        for (int q = 0; q < 10; ++q) {
            const double y = __shfl_down_sync(0xffffffffu, v[q], o2);
            v[q] = (q >= 4 && q <= 6) ? fmax(v[q], y) : v[q] + y;
        }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0)
        for (int q = 0; q < 10; ++q) red[warp][q] = v[q];
    __syncthreads();
    if (threadIdx.x == 0)
        for (int q = 0; q < 10; ++q) {
            double t = red[0][q];
            for (int w = 1; w < NT / 32; ++w) t = (q >= 4 && q <= 6) ? fmax(t, red[w][q]) : t + red[w][q];
            o[q] = t;
        }
    __syncthreads();
}

// Record, time and next dt of batch instance `inst` from its reduced diagnostics o[10]
// (one thread).
template <class Real>
__device__ __forceinline__ void batch_finish_inst(const Inst<Real>& I, int inst, const double* o,
                                                  double* __restrict__ idt, double* __restrict__ it,
                                                  double* __restrict__ irec, int kick, Control* ctl) {
    const double dt = idt[inst];
    if (kick) it[inst] += dt;
    double* rec = irec + (size_t)inst * DIAG_N;
    rec[0] = it[inst];
    rec[1] = kick ? dt : 0.0;
    rec[2] = o[3];
    rec[3] = sqrt(o[4]);
    rec[4] = o[0];
    rec[5] = o[1];
    rec[6] = o[2];
    rec[7] = sqrt(o[5]);
    rec[8] = o[7];
    rec[9] = o[8];
    rec[10] = rec[10] + (kick ? 1.0 : 0.0);
    rec[11] = 0.0;
    rec[12] = o[9];
    if (o[6] != 0.0) atomicOr(&ctl->status, ST_NONFINITE);
    idt[inst] = next_dt(I.C, rec[3], rec[7]);
}

// Batch instance `inst` in one block (the persistent step): its whole segment.
template <class Real, int NT>
__device__ __forceinline__ void batch_reduce_inst(const ParticleSet& S,
                                                  const uint32_t* __restrict__ pcount,
                                                  const uint32_t* __restrict__ off,
                                                  const Inst<Real>& I, int inst, int dim,
                                                  double* __restrict__ idt, double* __restrict__ it,
                                                  double* __restrict__ irec, int kick, Control* ctl,
                                                  double (*red)[10]) {
    double o[10];
    batch_partial<NT>(S, pcount, off[I.cell_base], off[I.cell_base_end], dim, o, red);
    if (threadIdx.x == 0) batch_finish_inst<Real>(I, inst, o, idt, it, irec, kick, ctl);
    __syncthreads();
}

}  // namespace sph
