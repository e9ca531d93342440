// Per-instance reduction of a batched step: the diagnostics of an instance's contiguous
// cell-order segment (block partials, then a fixed-order combination) and the instance's
// record, time and next dt (Sec. 2.1 step control). Used by the per-phase batch kernels
// (batch.cu) and the persistent step kernel.
#pragma once

#include "reduce_impl.cuh"

namespace sph {

// Finiteness from the exponent bits (integer pipe; isfinite compares on the FP64 pipe,
// which runs at 1/64 of the FP32 rate on this part).
__device__ __forceinline__ bool finite_bits(double v) {
    return ((unsigned long long)__double_as_longlong(v) & 0x7ff0000000000000ull) !=
           0x7ff0000000000000ull;
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
            bad |= !finite_bits(rho);
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
        bool bk = !finite_bits(rho);
#pragma unroll
        for (int d = 0; d < 3; ++d)
            if (d < dim) {
                u2 += u[d] * u[d];
                a2 += a[d] * a[d];
                bk |= !finite_bits(u[d]) || !finite_bits(x[d]);
            }
        bk |= !finite_bits(a2);
        px += m * u[0];
        py += m * u[1];
        if (dim == 3) pz += m * u[2];
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

// First stage of the two-stage reduction (one block of NT threads): chunk `chunk_id` of
// BATCH_SPLIT consecutive chunks of instance `inst`'s cell-order segment, its partials to
// part[(inst * BATCH_SPLIT + chunk_id) * 10 ...].
template <class Real, int NT>
__device__ __forceinline__ void batch_chunk_partials(const ParticleSet& S,
                                                     const uint32_t* __restrict__ pcount,
                                                     const uint32_t* __restrict__ off,
                                                     const Inst<Real>& I, int inst, int chunk_id,
                                                     int dim, double* __restrict__ part,
                                                     double (*red)[10]) {
    const uint32_t b0 = off[I.cell_base], e0 = off[I.cell_base_end];
    const uint32_t chunk = (e0 - b0 + BATCH_SPLIT - 1) / BATCH_SPLIT;
    const uint32_t b = b0 + chunk_id * chunk;
    const uint32_t e = b + chunk < e0 ? b + chunk : e0;
    double o[10];
    batch_partial<NT>(S, pcount, b < e0 ? b : e0, b < e0 ? e : e0, dim, o, red);
    if (threadIdx.x == 0)
        for (int q = 0; q < 10; ++q) part[((size_t)inst * BATCH_SPLIT + chunk_id) * 10 + q] = o[q];
}

// Second stage (one warp, every lane calls it): instance `inst`'s BATCH_SPLIT partials
// combined by a fixed shuffle tree, then its record, time and next dt.
template <class Real>
__device__ __forceinline__ void batch_finish_warp(const Inst<Real>& I, int inst,
                                                  const double* __restrict__ part,
                                                  double* __restrict__ idt, double* __restrict__ it,
                                                  double* __restrict__ irec, int kick, Control* ctl) {
    const int lane = threadIdx.x & 31;
    double v[10];
    for (int q = 0; q < 10; ++q)
        v[q] = lane < BATCH_SPLIT ? part[((size_t)inst * BATCH_SPLIT + lane) * 10 + q] : 0.0;
    for (int o2 = 16; o2 > 0; o2 >>= 1)
        for (int q = 0; q < 10; ++q) {
            const double y = __shfl_down_sync(0xffffffffu, v[q], o2);
            v[q] = (q >= 4 && q <= 6) ? fmax(v[q], y) : v[q] + y;
        }
    if (lane == 0) batch_finish_inst<Real>(I, inst, v, idt, it, irec, kick, ctl);
}

}  // namespace sph
