// Host-side launchers of the device kernels (internal to the library).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <string>

#include "sph_device.cuh"

namespace sph {

// nnps.cu (the build stages take the instance table of a StepLaunch, declared below)
int radix_passes(int ncells);
size_t radix_hist_words(int n);
int launch_radix_sort(uint32_t* keys[2], uint32_t* vals[2], int n, int passes, uint32_t* hist,
                      Control* ctl, cudaStream_t st);
void launch_cell_offsets(const uint32_t* skeys, int n, int ncells, uint32_t* off, Control* ctl,
                         cudaStream_t st, int sms);
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

// batch.cu: constants of one instance of a batch (device table, one entry per instance).
template <class Real>
struct Inst {
    Grid G;
    PairConst<Real> K;
    StepConst C;
    uint32_t cell_base;      // first global cell id of the instance
    uint32_t cell_base_end;  // first global cell id of the next instance
};
// Everything one step's kernels need. A single problem is a table of one instance whose
// dt is the control block's; a batch has one entry per instance.
struct StepLaunch {
    int precision, dim, kernel, n, sms, ninst, kick, maxn;
    int group_d, group_m, grid_d, grid_m;  // lanes per destination and grid of each pass
    int finalize;                 // 1: the momentum pass reduces the diagnostics (single)
    const void* tab;              // Inst<Real>[ninst]
    const void* tab_host;         // single problem: host copy of its entry (passed by value), else null
    const uint32_t* id_bounds;    // ninst + 1 global-id bounds
    const uint32_t* cell_bounds;  // ninst + 1 global-cell bounds
    double* idt;                  // dt of the next step, per instance
    double* it;                   // batch: time per instance
    double* irec;                 // batch: diagnostics per instance
    ParticleSet Sin;              // current set (drift, reorder source)
    ParticleSet S;                // cell-ordered set (reorder target, pair passes)
    void* P;
    void* Q;
    void* R;
    void* E;                      // FP32 pair loops: position residuals (reorder_one)
    int edac;                     // the EDAC form: the reorder gathers the pressure state
    const uint32_t* skeys;
    const uint32_t* off;
    uint32_t* nl;                 // neighbour list, nl[k * n + i], k < maxn
    uint32_t* cnt;                // list length per particle
    uint32_t* pcount;             // batch: interacting pairs and candidates per particle
    double* bpart;                // batch: BATCH_SPLIT x 10 partial diagnostics per instance
    double* pm;                   // single: 8 doubles per momentum block
    double* pd;                   // single: 4 doubles per density block
    double* cpart;                // single: 8 doubles per chunk of destinations (momentum, one lane)
    int dyn;                      // one-lane passes taking chunks from a counter: 1 density (single
                                  // problems), 2 momentum (problems with walls)
    double* history;
    Control* ctl;
};
void launch_drift_keys(const StepLaunch& L, int drift, uint32_t* keys, cudaStream_t st);
// Gather into cell order (reorder + EOS shadow) and the cell table off[0..ncells].
void launch_reorder(const StepLaunch& L, const uint32_t* perm, int carry_rates, uint32_t* off,
                    int ncells, uint32_t* work, int work_words, cudaStream_t st);
// Sort workspace (digit histograms, tile counters, look-back words) in 32-bit words.
size_t sort_work_words(int n, int passes);
void launch_keys_hist(const StepLaunch& L, int drift, uint32_t* keys0, int passes, uint32_t* work,
                      cudaStream_t st);
int launch_onesweep(int n, uint32_t* keys[2], uint32_t* vals[2], int passes, uint32_t* work,
                    Control* ctl, unsigned long long wait_ns, cudaStream_t st);
int pair_threads();
void launch_pairs(const StepLaunch& L, cudaStream_t st);
void launch_density_pass(const StepLaunch& L, cudaStream_t st);
void launch_momentum_pass(const StepLaunch& L, cudaStream_t st);
// Solid-wall pressure (scheme option) between the density and the momentum pass.
void launch_wall_pressure(const StepLaunch& L, cudaStream_t st);
constexpr int BATCH_SPLIT = 32;  // blocks per instance in the first stage of a batch reduction
void launch_batch_reduce(const StepLaunch& L, cudaStream_t st);
// fused_f32.cu / fused_f64.cu: the whole step as one cooperative launch (persistent blocks,
// grid barriers between the phases).
constexpr int FUSED_THREADS = 256;  // = the radix: one digit per thread in the sort phases
constexpr int FUSED_PART = 16;      // doubles of per-block partials
struct FusedLaunch {
    StepLaunch L;                // L.Sin: current set; L.S: the other set (reorder target)
    uint32_t* keys[2];
    uint32_t* vals[2];
    uint32_t* work;              // one-sweep sort workspace (zero at launch; zeroed again)
    int work_words;
    uint32_t* off;               // cell table, written by the reorder phase
    double* part;                // FUSED_PART doubles per block
    int passes, ntiles, ncells;
    int wall_pass;               // the solid-wall pressure phase runs between the pair passes
    unsigned long long wait_ns;  // limit of one barrier wait
};
cudaError_t launch_fused(const FusedLaunch& F, int T, int grid, cudaStream_t st);
int fused_max_blocks_per_sm(int precision, int dim, int kernel, int T);
int radix_tiles(int n);

// pass 0: density (thread per destination), 1: momentum (T = 1, 2, 4 or 8 lanes per
// destination)
// single: the single-problem form of the kernels (constants by value), else the batch form
int pairs_max_blocks_per_sm(int precision, int pass, int dim, int kernel, int T, int single);

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
    int precision, dim, kernel, n, sms, kick;
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
    const uint32_t* nl;    // taped neighbour list of the evaluation (nl[k * n + i])
    const uint32_t* cnt;
    double* part;
    AdjCtl* actl;
};
void launch_adjoint_eval(const AdjLaunch& A, const PairConst<float>& Kf, const PairConst<double>& Kd,
                         cudaStream_t st);
void launch_adjoint_scatter(const AdjLaunch& A, const AdjSet& out, cudaStream_t st);
void launch_tape_list(const uint32_t* nl, const uint32_t* cnt, int n, uint32_t* tnl, uint32_t* tcnt,
                      int sms, cudaStream_t st);
void launch_adjoint_terminal(const AdjSet& L, const ParticleSet& S, int n, int dim, int sms,
                             cudaStream_t st);
void launch_adjoint_to_original(const AdjLaunch& A, double* out, cudaStream_t st);
int adjoint_partial_blocks(int n, int sms);

}  // namespace sph
