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
// px py pz ke max|u|^2 max|a|^2 bad pairs candidates wall-pairs. Only the momentum and
// kinetic-energy sums use the FP64 pipe (1/64 of the FP32 rate on this part): counts,
// flags and maxima (the bit pattern of a non-negative double orders like the double)
// reduce as integers, as in the single-problem reduction.
template <int NT>
__device__ __forceinline__ void batch_partial(const ParticleSet& S,
                                              const uint32_t* __restrict__ pcount, uint32_t b,
                                              uint32_t e, int dim, double* o, double (*red)[10]) {
    double px = 0, py = 0, pz = 0, ke = 0;
    unsigned long long u2b = 0, a2b = 0, np = 0, nc = 0, nw = 0;
    unsigned bad = 0;
    for (uint32_t k = b + threadIdx.x; k < e; k += NT) {
        const bool fluid = !(S.tag[k] & WALL_BIT);
        const uint32_t pk = pcount[2 * (size_t)k], ck = pcount[2 * (size_t)k + 1];
        const double rho = S.rho[k];
        np += pk;
        nc += ck;
        if (!fluid) {
            nw += pk;
            bad |= !isfinite(rho);
            continue;
        }
        double u[3] = {0, 0, 0}, a[3] = {0, 0, 0}, x[3] = {0, 0, 0};
#pragma unroll
        for (int d = 0; d < 3; ++d)
            if (d < dim) {
                u[d] = S.u[d][k];
                a[d] = S.a[d][k];
                x[d] = S.x[d][k];
            }
        const double m = S.m[k];
        double u2 = 0, a2 = 0;
        bool bk = !isfinite(rho);
#pragma unroll
        for (int d = 0; d < 3; ++d)
            if (d < dim) {
                u2 += u[d] * u[d];
                a2 += a[d] * a[d];
                bk |= !isfinite(u[d]) || !isfinite(x[d]);
            }
        bk |= !isfinite(a2);
        px += m * u[0];
        py += m * u[1];
        pz += m * u[2];
        ke += 0.5 * m * u2;
        if (bk) bad = 1u;
        else {
            u2b = u2b > (unsigned long long)__double_as_longlong(u2) ? u2b
                                                                    : (unsigned long long)__double_as_longlong(u2);
            a2b = a2b > (unsigned long long)__double_as_longlong(a2) ? a2b
                                                                    : (unsigned long long)__double_as_longlong(a2);
        }
    }
#pragma unroll
    for (int o2 = 16; o2 > 0; o2 >>= 1) {
        px += __shfl_down_sync(0xffffffffu, px, o2);
        py += __shfl_down_sync(0xffffffffu, py, o2);
        pz += __shfl_down_sync(0xffffffffu, pz, o2);
        ke += __shfl_down_sync(0xffffffffu, ke, o2);
        const unsigned long long ou = __shfl_down_sync(0xffffffffu, u2b, o2);
        const unsigned long long oa = __shfl_down_sync(0xffffffffu, a2b, o2);
        u2b = u2b > ou ? u2b : ou;
        a2b = a2b > oa ? a2b : oa;
        np += __shfl_down_sync(0xffffffffu, np, o2);
        nc += __shfl_down_sync(0xffffffffu, nc, o2);
        nw += __shfl_down_sync(0xffffffffu, nw, o2);
        bad |= __shfl_down_sync(0xffffffffu, bad, o2);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        red[warp][0] = px;
        red[warp][1] = py;
        red[warp][2] = pz;
        red[warp][3] = ke;
        red[warp][4] = __longlong_as_double((long long)u2b);
        red[warp][5] = __longlong_as_double((long long)a2b);
        red[warp][6] = bad ? 1.0 : 0.0;
        red[warp][7] = (double)np;
        red[warp][8] = (double)nc;
        red[warp][9] = (double)nw;
    }
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
