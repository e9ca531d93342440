// Host-side launchers of the device kernels (internal to the library).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <string>

#include "sph_device.cuh"

namespace sph {

// nnps.cu
void launch_drift_keys(const ParticleSet& S, int n, const Grid& G, const StepConst& C,
                       Control* ctl, int drift, uint32_t* keys, cudaStream_t st, int sms);
int radix_passes(int ncells);
size_t radix_hist_words(int n);
int launch_radix_sort(uint32_t* keys[2], uint32_t* vals[2], int n, int passes, uint32_t* hist,
                      Control* ctl, cudaStream_t st);
void launch_cell_offsets(const uint32_t* skeys, int n, int ncells, uint32_t* off, Control* ctl,
                         cudaStream_t st, int sms);
void launch_reorder(int precision, const ParticleSet& in, const ParticleSet& out,
                    const uint32_t* perm, int n, int dim, const StepConst& C, Control* ctl,
                    int kick, int carry_rates, void* P, void* Q, void* R, cudaStream_t st, int sms);
void launch_gather_by_id(const double* field, const uint32_t* tag, int n, uint32_t first,
                         uint32_t count, double* out, cudaStream_t st, int sms);
void launch_scatter_by_id(double* field, const uint32_t* tag, int n, uint32_t first,
                          uint32_t count, const double* in, cudaStream_t st, int sms);
void launch_cell_of_by_id(const uint32_t* skeys, const uint32_t* tag, int n, uint32_t* cell_of,
                          int64_t* order, cudaStream_t st, int sms);
void launch_wrap_all(const ParticleSet& S, int n, const Grid& G, cudaStream_t st, int sms);
void launch_export_neighbors(int precision, int dim, const void* P, const uint32_t* skeys,
                             const uint32_t* off, const uint32_t* tag, int n, const Grid& G,
                             const PairConst<float>& Kf, const PairConst<double>& Kd, int pass,
                             uint32_t* counts, const int64_t* row_off, int32_t* idx,
                             cudaStream_t st, int sms);

// capi.cu: sets the message sph_last_error(NULL) returns on this thread
void set_global_error(const std::string& msg);

// pairs.cu: one evaluation = density pass (group size group_d, grid_d blocks) then
// momentum pass (group_m, grid_m). pm / pd: per-block partials of the two passes.
struct PairLaunch {
    int precision, dim, kernel, kick, n;
    int group_d, group_m, grid_d, grid_m;
    const void* P;
    void* Q;
    void* R;
    const uint32_t* skeys;
    const uint32_t* off;
    Grid G;
    StepConst C;
    ParticleSet S;
    Control* ctl;
    uint32_t* nl;   // neighbour list, nl[k * n + i], k < maxn
    uint32_t* cnt;  // list length per particle
    int maxn;
    double* pm;  // 8 doubles per momentum block
    double* pd;  // 4 doubles per density block
    double* history;
};
int pair_threads();
void launch_pairs(const PairLaunch& L, const PairConst<float>& Kf, const PairConst<double>& Kd,
                  cudaStream_t st);
void launch_density_pass(const PairLaunch& L, const PairConst<float>& Kf,
                         const PairConst<double>& Kd, cudaStream_t st);
void launch_momentum_pass(const PairLaunch& L, const PairConst<float>& Kf,
                          const PairConst<double>& Kd, cudaStream_t st);
// pass 0: density (thread per destination), 1: momentum (T = 1, 2, 4 or 8 lanes per
// destination)
int pairs_max_blocks_per_sm(int precision, int pass, int dim, int kernel, int T);

// adjoint.cu: adjoint state (FP64, cell order of the current evaluation)
struct AdjSet {
    double* x[3];
    double* u[3];
    double* rho;
    double* a[3];
    double* xs[3];
};
struct AdjCtl {
    double g_nu, g_alpha;  // running d KE / d nu, d KE / d alpha
    unsigned ticket;
};
// One reversed evaluation on a taped configuration (P, Q, R after its density pass).
struct AdjLaunch {
    int precision, dim, kernel, n, sms, kick, maxn;
    double dt;
    const void* P;
    const void* Q;
    const void* R;
    const uint32_t* perm;  // taped order -> previous order
    const uint32_t* tag;   // taped order
    Grid G;
    StepConst C;
    AdjSet L;              // cotangents in the taped order (in: state, out: += x)
    double* luh[3];        // lambda of the evaluation velocities
    double* rhom;
    double* lrho_tot;
    void* CA;
    void* CS;
    uint32_t* keys;
    uint32_t* off;
    uint32_t* nl;
    uint32_t* cnt;
    double* part;
    AdjCtl* actl;
    Control* ctl;
};
void launch_adjoint_eval(const AdjLaunch& A, const PairConst<float>& Kf, const PairConst<double>& Kd,
                         cudaStream_t st);
void launch_adjoint_scatter(const AdjLaunch& A, const AdjSet& out, cudaStream_t st);
void launch_adjoint_terminal(const AdjSet& L, const ParticleSet& S, int n, int dim, int sms,
                             cudaStream_t st);
void launch_adjoint_to_original(const AdjLaunch& A, double* out, cudaStream_t st);
int adjoint_partial_blocks(int n, int sms);

}  // namespace sph
