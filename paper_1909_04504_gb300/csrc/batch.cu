// Per-instance reduction of a batched step. A batch holds many independent problems
// (instances) of uneven size in one set of arrays; the sort key is the instance's first
// global cell id plus the local cell id, so a stable sort keeps every instance contiguous
// and, inside it, in the order a single run of that instance would have. The step kernels
// are the single-problem kernels (they read every constant from the instance table), so
// an instance of a batch computes bitwise what its single run computes.
#include "sph_device.cuh"
#include "sph_launch.h"

namespace sph {

// One block per instance over its contiguous cell-order segment: FP64 diagnostics in a
// fixed order, the record, the time, the next dt (fixed or the CFL-type criteria), status.
template <class Real>
__global__ void __launch_bounds__(256)
k_batch_reduce(ParticleSet S, const uint32_t* __restrict__ pcount, const uint32_t* __restrict__ off,
               const Inst<Real>* __restrict__ tab, int ninst, int dim, double* __restrict__ idt,
               double* __restrict__ it, double* __restrict__ irec, int kick, Control* ctl) {
    __shared__ double red[8][10];
    if (ctl->status) return;
    const int inst = blockIdx.x;
    if (inst >= ninst) return;
    const Inst<Real>& I = tab[inst];
    const uint32_t b = off[I.cell_base], e = off[I.cell_base_end];
    double v[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};  // px py pz ke u2 a2 bad pairs cand wall
    for (uint32_t k = b + threadIdx.x; k < e; k += blockDim.x) {
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
    for (int o = 16; o > 0; o >>= 1)
        for (int q = 0; q < 10; ++q) {
            const double y = __shfl_down_sync(0xffffffffu, v[q], o);
            v[q] = (q >= 4 && q <= 6) ? fmax(v[q], y) : v[q] + y;
        }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0)
        for (int q = 0; q < 10; ++q) red[warp][q] = v[q];
    __syncthreads();
    if (threadIdx.x == 0) {
        double o[10];
        for (int q = 0; q < 10; ++q) {
            double t = red[0][q];
            for (int w = 1; w < (int)(blockDim.x / 32); ++w)
                t = (q >= 4 && q <= 6) ? fmax(t, red[w][q]) : t + red[w][q];
            o[q] = t;
        }
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
        double dn = I.C.dt_fixed;
        if (!(dn > 0.0)) {
            dn = 0.25 * I.C.h / (I.C.c0 + rec[3]);
            if (rec[7] > 0.0) dn = fmin(dn, 0.25 * sqrt(I.C.h / rec[7]));
            if (I.C.nu > 0.0) dn = fmin(dn, 0.125 * I.C.h * I.C.h / I.C.nu);
        }
        idt[inst] = dn;
    }
}

// ---------------------------------------------------------------- launchers
void launch_batch_reduce(const StepLaunch& L, cudaStream_t st) {
    if (L.precision)
        k_batch_reduce<float><<<L.ninst, 256, 0, st>>>(L.S, L.pcount, L.off, (const Inst<float>*)L.tab,
                                                       L.ninst, L.dim, L.idt, L.it, L.irec, L.kick,
                                                       L.ctl);
    else
        k_batch_reduce<double><<<L.ninst, 256, 0, st>>>(L.S, L.pcount, L.off,
                                                        (const Inst<double>*)L.tab, L.ninst, L.dim,
                                                        L.idt, L.it, L.irec, L.kick, L.ctl);
}

}  // namespace sph
