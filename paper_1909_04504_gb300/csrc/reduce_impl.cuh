// End-of-evaluation bookkeeping (Sec. 2.1 step control): the diagnostics record, the
// history entry, the time, the next dt (fixed, or the CFL-type criteria) and the status of
// a single problem, from already reduced totals. Shared by the per-phase kernels and the
// persistent step kernel (the per-instance reduction of a batch is in batch_impl.cuh).
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

}  // namespace sph
