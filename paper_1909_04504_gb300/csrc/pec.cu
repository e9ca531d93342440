// Midpoint predict-evaluate-correct form of the predictor-corrector of Sec. 2.1 (after
// Monaghan 2005; scheme option SPH_INTEGRATOR_PEC). One step from (x^n, u^n, rho^n) with
// the rates of the evaluation at t^n:
//   predictor   u* = u^n + dt/2 a^n,  x* = wrap(x^n + dt/2 (u^n + xsph^n)),
//               rho* = rho^n + dt/2 arho^n;
//   neighbour build and evaluation at (x*, u*, rho*);
//   corrector   u^{n+1} = u^n + dt a*,  x^{n+1} = wrap(x^n + dt (u^n + dt/2 a* + xsph*)),
//               rho^{n+1} = rho^n + dt arho*;
//   neighbour build and evaluation at t^{n+1} (diagnostics, next dt).
// Walls keep x and u; their density is integrated like the fluid's. With summation
// density the evaluations set rho and neither stage touches it. The two stages are plain
// streaming kernels (one thread per particle, FP64); the builds and evaluations are the
// kernels of the kick-drift-kick step, run without their kicks.
#include "pec.h"
#include "step_impl.cuh"

namespace sph {

namespace {

constexpr int PEC_THREADS = 256;

// Periodic wrap of coordinate d into [lo, hi) (Sec. 3 update_domain), with the rounding
// of the drift kernel.
__device__ __forceinline__ double pec_wrap(double x, const Grid& G, int d) {
    if (!G.periodic[d] || (x >= G.lo[d] && x < G.hi[d])) return x;
    const double k = floor(__ddiv_rn(__dsub_rn(x, G.lo[d]), G.L[d]));
    x = __dsub_rn(x, __dmul_rn(k, G.L[d]));
    if (x >= G.hi[d]) x = __dsub_rn(x, G.L[d]);
    if (x < G.lo[d]) x = G.lo[d];
    return x;
}

// Predictor of particle i (current order): saves x, u, rho and advances to the half step.
template <int DIM>
__device__ __forceinline__ void pec_predict_one(const ParticleSet& S, double* __restrict__ save,
                                                int n, int i, const Grid& G, double dt,
                                                int continuity) {
    // every load before any store (the state arrays could alias as far as the compiler
    // knows)
    const double hdt = 0.5 * dt;
    const bool fluid = !(S.tag[i] & WALL_BIT);
    double x[DIM], u[DIM], a[DIM], xs[DIM];
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
        x[d] = S.x[d][i];
        u[d] = S.u[d][i];
        a[d] = S.a[d][i];
        xs[d] = S.xs[d][i];
    }
    const double rho = S.rho[i];
    const double arho = S.arho[i];
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
        save[(size_t)d * n + i] = x[d];
        save[(size_t)(DIM + d) * n + i] = u[d];
    }
    save[(size_t)(2 * DIM) * n + i] = rho;
    if (fluid)
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            S.u[d][i] = u[d] + hdt * a[d];
            S.x[d][i] = pec_wrap(x[d] + hdt * (u[d] + xs[d]), G, d);
        }
    if (continuity) S.rho[i] = rho + hdt * arho;
}

// Corrector of particle k (midpoint order), whose saved state sits at position o.
template <int DIM>
__device__ __forceinline__ void pec_correct_one(const ParticleSet& S, const double* __restrict__ save,
                                                int n, int k, uint32_t o, const Grid& G, double dt,
                                                int continuity) {
    const double hdt = 0.5 * dt;
    const bool fluid = !(S.tag[k] & WALL_BIT);
    double x0[DIM], u0[DIM], a[DIM], xs[DIM];
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
        x0[d] = save[(size_t)d * n + o];
        u0[d] = save[(size_t)(DIM + d) * n + o];
        a[d] = S.a[d][k];
        xs[d] = S.xs[d][k];
    }
    const double rho0 = save[(size_t)(2 * DIM) * n + o];
    const double arho = S.arho[k];
    if (fluid)
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            const double ubar = u0[d] + hdt * a[d];
            S.x[d][k] = pec_wrap(x0[d] + dt * (ubar + xs[d]), G, d);
            S.u[d][k] = u0[d] + dt * a[d];
        }
    if (continuity) S.rho[k] = rho0 + dt * arho;
}

template <int DIM>
__global__ void __launch_bounds__(PEC_THREADS)
k_pec_predict(ParticleSet S, double* __restrict__ save, int n, Grid G,
              const double* __restrict__ idt, double* __restrict__ dt_step, int continuity,
              const Control* ctl) {
    if (ctl->status) return;
    const double dt = *idt;
    if (blockIdx.x == 0 && threadIdx.x == 0) *dt_step = dt;
    for (int i = blockIdx.x * PEC_THREADS + (int)threadIdx.x; i < n; i += gridDim.x * PEC_THREADS)
        pec_predict_one<DIM>(S, save, n, i, G, dt, continuity);
}

template <int DIM>
__global__ void __launch_bounds__(PEC_THREADS)
k_pec_correct(ParticleSet S, const double* __restrict__ save, const uint32_t* __restrict__ perm,
              int n, Grid G, const double* __restrict__ dt_step, int continuity,
              const Control* ctl) {
    if (ctl->status) return;
    const double dt = *dt_step;
    for (int k = blockIdx.x * PEC_THREADS + (int)threadIdx.x; k < n; k += gridDim.x * PEC_THREADS) {
        const uint32_t o = perm[k];
        if (o >= (uint32_t)n) continue;  // a completed build gives a permutation of [0, n)
        pec_correct_one<DIM>(S, save, n, k, o, G, dt, continuity);
    }
}

// Batch forms: the instance of a particle from its cell key, its grid and step size from
// the instance table (dt_step holds one step size per instance).
template <class Real, int DIM>
__global__ void __launch_bounds__(PEC_THREADS)
k_pec_predict_batch(ParticleSet S, double* __restrict__ save, int n,
                    const Inst<Real>* __restrict__ tab, const uint32_t* __restrict__ cell_bounds,
                    int ninst, const uint32_t* __restrict__ skeys, const double* __restrict__ idt,
                    double* __restrict__ dt_step, int continuity, const Control* ctl) {
    if (ctl->status) return;
    const int stride = gridDim.x * PEC_THREADS;
    const int tid = blockIdx.x * PEC_THREADS + (int)threadIdx.x;
    for (int q = tid; q < ninst; q += stride) dt_step[q] = idt[q];
    for (int i = tid; i < n; i += stride) {
        const int inst = find_instance(cell_bounds, ninst, skeys[i]);
        pec_predict_one<DIM>(S, save, n, i, tab[inst].G, idt[inst], continuity);
    }
}

template <class Real, int DIM>
__global__ void __launch_bounds__(PEC_THREADS)
k_pec_correct_batch(ParticleSet S, const double* __restrict__ save,
                    const uint32_t* __restrict__ perm, int n, const Inst<Real>* __restrict__ tab,
                    const uint32_t* __restrict__ cell_bounds, int ninst,
                    const uint32_t* __restrict__ skeys, const double* __restrict__ dt_step,
                    int continuity, const Control* ctl) {
    if (ctl->status) return;
    for (int k = blockIdx.x * PEC_THREADS + (int)threadIdx.x; k < n; k += gridDim.x * PEC_THREADS) {
        const uint32_t o = perm[k];
        if (o >= (uint32_t)n) continue;
        const int inst = find_instance(cell_bounds, ninst, skeys[k]);
        pec_correct_one<DIM>(S, save, n, k, o, tab[inst].G, dt_step[inst], continuity);
    }
}

__global__ void k_pec_record(Control* ctl, double* __restrict__ history,
                             const double* __restrict__ dt_step) {
    // a non-finite value found by the last evaluation still ends the step (the state is
    // that of the step where it appeared); any other status stopped the step part-way
    if (ctl->status & ~ST_NONFINITE) return;
    const double dt = *dt_step;
    ctl->t += dt;
    ctl->step += 1;
    double* rec = ctl->rec;
    rec[0] = ctl->t;
    rec[1] = dt;
    rec[10] = (double)ctl->step;
    double* h = history + (size_t)(ctl->hist_count % HIST_CAP) * DIAG_N;
    for (int k = 0; k < DIAG_N; ++k) h[k] = rec[k];
    ctl->hist_count += 1;
    __threadfence();
}

// Batch: per instance, t and the step count advance by the step just taken (the
// reductions of the end-of-step evaluation wrote the rest of the record).
__global__ void k_pec_record_batch(double* __restrict__ it, double* __restrict__ irec,
                                   const double* __restrict__ dt_step, int ninst,
                                   const Control* ctl) {
    if (ctl->status & ~ST_NONFINITE) return;
    for (int q = blockIdx.x * blockDim.x + (int)threadIdx.x; q < ninst; q += gridDim.x * blockDim.x) {
        const double dt = dt_step[q];
        it[q] += dt;
        double* rec = irec + (size_t)q * DIAG_N;
        rec[0] = it[q];
        rec[1] = dt;
        rec[10] += 1.0;
    }
}

int stage_grid(int n, int sms) {
    const long long want = ((long long)n + PEC_THREADS - 1) / PEC_THREADS;
    const long long cap = (long long)sms * 8;
    return (int)(want < 1 ? 1 : (want > cap ? cap : want));
}

}  // namespace

void launch_pec_predict(const ParticleSet& S, double* save, int n, int dim, const Grid& G,
                        const double* idt, double* dt_step, int continuity, const Control* ctl,
                        int sms, cudaStream_t st) {
    const int g = stage_grid(n, sms);
    if (dim == 3) k_pec_predict<3><<<g, PEC_THREADS, 0, st>>>(S, save, n, G, idt, dt_step, continuity, ctl);
    else k_pec_predict<2><<<g, PEC_THREADS, 0, st>>>(S, save, n, G, idt, dt_step, continuity, ctl);
}

void launch_pec_correct(const ParticleSet& S, const double* save, const uint32_t* perm, int n,
                        int dim, const Grid& G, const double* dt_step, int continuity,
                        const Control* ctl, int sms, cudaStream_t st) {
    const int g = stage_grid(n, sms);
    if (dim == 3)
        k_pec_correct<3><<<g, PEC_THREADS, 0, st>>>(S, save, perm, n, G, dt_step, continuity, ctl);
    else k_pec_correct<2><<<g, PEC_THREADS, 0, st>>>(S, save, perm, n, G, dt_step, continuity, ctl);
}

void launch_pec_record(Control* ctl, double* history, const double* dt_step, cudaStream_t st) {
    k_pec_record<<<1, 1, 0, st>>>(ctl, history, dt_step);
}

template <class Real>
static void predict_batch_t(const ParticleSet& S, double* save, int n, int dim, const void* tab,
                            const uint32_t* cell_bounds, int ninst, const uint32_t* skeys,
                            const double* idt, double* dt_step, int continuity, const Control* ctl,
                            int g, cudaStream_t st) {
    const Inst<Real>* T = (const Inst<Real>*)tab;
    if (dim == 3)
        k_pec_predict_batch<Real, 3><<<g, PEC_THREADS, 0, st>>>(S, save, n, T, cell_bounds, ninst,
                                                                skeys, idt, dt_step, continuity, ctl);
    else
        k_pec_predict_batch<Real, 2><<<g, PEC_THREADS, 0, st>>>(S, save, n, T, cell_bounds, ninst,
                                                                skeys, idt, dt_step, continuity, ctl);
}

template <class Real>
static void correct_batch_t(const ParticleSet& S, const double* save, const uint32_t* perm, int n,
                            int dim, const void* tab, const uint32_t* cell_bounds, int ninst,
                            const uint32_t* skeys, const double* dt_step, int continuity,
                            const Control* ctl, int g, cudaStream_t st) {
    const Inst<Real>* T = (const Inst<Real>*)tab;
    if (dim == 3)
        k_pec_correct_batch<Real, 3><<<g, PEC_THREADS, 0, st>>>(S, save, perm, n, T, cell_bounds,
                                                                ninst, skeys, dt_step, continuity, ctl);
    else
        k_pec_correct_batch<Real, 2><<<g, PEC_THREADS, 0, st>>>(S, save, perm, n, T, cell_bounds,
                                                                ninst, skeys, dt_step, continuity, ctl);
}

void launch_pec_predict_batch(const ParticleSet& S, double* save, int n, int dim, int precision,
                              const void* tab, const uint32_t* cell_bounds, int ninst,
                              const uint32_t* skeys, const double* idt, double* dt_step,
                              int continuity, const Control* ctl, int sms, cudaStream_t st) {
    const int g = stage_grid(n > ninst ? n : ninst, sms);
    if (precision) predict_batch_t<float>(S, save, n, dim, tab, cell_bounds, ninst, skeys, idt, dt_step, continuity, ctl, g, st);
    else predict_batch_t<double>(S, save, n, dim, tab, cell_bounds, ninst, skeys, idt, dt_step, continuity, ctl, g, st);
}

void launch_pec_correct_batch(const ParticleSet& S, const double* save, const uint32_t* perm, int n,
                              int dim, int precision, const void* tab, const uint32_t* cell_bounds,
                              int ninst, const uint32_t* skeys, const double* dt_step,
                              int continuity, const Control* ctl, int sms, cudaStream_t st) {
    const int g = stage_grid(n, sms);
    if (precision) correct_batch_t<float>(S, save, perm, n, dim, tab, cell_bounds, ninst, skeys, dt_step, continuity, ctl, g, st);
    else correct_batch_t<double>(S, save, perm, n, dim, tab, cell_bounds, ninst, skeys, dt_step, continuity, ctl, g, st);
}

void launch_pec_record_batch(double* it, double* irec, const double* dt_step, int ninst,
                             const Control* ctl, cudaStream_t st) {
    k_pec_record_batch<<<(ninst + 127) / 128, 128, 0, st>>>(it, irec, dt_step, ninst, ctl);
}

}  // namespace sph
