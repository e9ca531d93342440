// Host runtime and C ABI (include/sph.h): context, device arena, the per-step launch
// sequence (Sec. 2.1 one_timestep: compute accelerations after a neighbour update, stage,
// update_domain), CUDA-graph capture of a step, state I/O and the debug exports.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "sph.h"
#include "sph_device.cuh"
#include "sph_launch.h"
#include "pec.h"
#include "sort_impl.cuh"

using namespace sph;

namespace {

thread_local std::string g_create_error;

constexpr double PI = 3.14159265358979323846;
constexpr uint32_t STATE_MAGIC = 0x53504853u;  // "SPHS"
constexpr uint32_t STATE_VERSION = 3;
constexpr int STATE_FIELDS = 16;  // FP64 arrays of a particle set (state_fields)

struct StateHeader {
    uint32_t magic, version;
    int64_t n;
    int32_t dim, precision, have_rates, cur;
    double t, dt;
    unsigned long long step;
    sph_scheme scheme;
};

}  // namespace

// The FP64 arrays of a particle set in the order of the saved state: x, u, rho, m, the
// rates (arho, a, xsph) and the EDAC pressure.
void state_fields(const ParticleSet& S, double** f) {
    double* t[STATE_FIELDS] = {S.x[0], S.x[1], S.x[2], S.u[0], S.u[1], S.u[2], S.rho, S.m,
                               S.arho, S.a[0], S.a[1], S.a[2], S.xs[0], S.xs[1], S.xs[2], S.p};
    for (int k = 0; k < STATE_FIELDS; ++k) f[k] = t[k];
}

struct sph_ctx {
    int device = 0;
    int sms = 1;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    sph_alloc_fn alloc = nullptr;
    sph_free_fn free_fn = nullptr;
    void* user = nullptr;
    std::string err;

    sph_domain dom{};
    Grid G{};
    int N = 0;
    int nwall = 0;                 // wall particles
    bool wall_pass = false;        // the scheme(s) in use take the solid-wall pressure pass
    bool pec = false;              // the scheme in use takes the midpoint integrator
    bool edac = false;             // the scheme in use is the EDAC form (pressure state)
    int pec_cont = 1;              // ... with the continuity density (else summation)
    double* pec_save = nullptr;    // midpoint integrator: saved (x, u, rho) + the step size
    uint32_t* perm = nullptr;      // sorted values of the last build: previous position
    std::vector<int64_t> arr_off;  // n_arrays + 1
    int passes = 1;

    // device arena
    void* arena = nullptr;
    size_t arena_bytes = 0;
    ParticleSet set[2]{};
    int cur = 0;
    void* P = nullptr;
    void* Q = nullptr;
    void* R = nullptr;
    void* E = nullptr;  // FP32 pair loops: residuals of the rounded positions
    uint32_t* keys[2]{};
    uint32_t* vals[2]{};
    uint32_t* skeys = nullptr;
    uint32_t* off = nullptr;
    uint32_t* hist = nullptr;
    double* pm = nullptr;  // momentum-pass block partials (8 doubles per block)
    double* pd = nullptr;     // density-pass block partials (4 doubles per block)
    double* cpart = nullptr;  // momentum chunk partials (single problem, one lane)
    Control* ctl = nullptr;
    double* history = nullptr;
    void* io = nullptr;  // scratch for get/set/exports: 4 N + 2 (8 N + 8) bytes, 256-aligned parts
    int grid_cap = 1;                 // largest pair-pass grid (sizes pm, pd)
    int bps[2][4] = {{1, 1, 1, 1}, {1, 1, 1, 1}};  // blocks per SM: [pass][T = 1, 2, 4, 8]
    int group_d = 1, group_m = 1;     // lanes per destination of the pair passes (equal)
    int grid_d = 1, grid_m = 1;
    uint32_t* nl = nullptr;           // neighbour list nl[k * N + i], separately allocated
    uint32_t* cnt = nullptr;          // list length per particle (arena)
    int maxn = 0;                     // list capacity per particle

    bool have_rates = false;
    bool nbr_valid = false;
    sph_scheme rates_scheme{};
    unsigned hist_at_call = 0;

    unsigned steps_total = 0;  // steps enqueued since creation / the last load (history index)

    // phase timing events (recorded inside captured steps when enabled)
    bool timing = false;
    bool timed_step_ran = false;
    int step_mode = SPH_STEP_GRAPH;   // per-phase kernels in a graph, or one persistent launch
    int fused_bps[4] = {0, 0, 0, 0};  // persistent kernel: blocks per SM for T = 1, 2, 4, 8
    double* fpart = nullptr;          // persistent kernel: per-block partials
    uint32_t* sort_work = nullptr;    // one-sweep sort: histograms, counters, look-back words
    bool work_dirty = true;           // a build may have stopped before clearing sort_work
    double* bpart = nullptr;          // batch: partial diagnostics per instance
    unsigned long long wait_ns = 1000000000ull;  // limit of one device-side wait
    bool last_fused = false;          // the last step ran as one persistent launch
    cudaEvent_t ev[7] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};

    // batch of independent instances (ninst > 0)
    int ninst = 0;
    std::vector<sph_domain> doms;     // per instance
    std::vector<Grid> grids;          // per instance
    std::vector<uint32_t> id_bounds_h, cell_bounds_h;
    void* d_tab = nullptr;            // Inst<Real>[ninst]
    uint32_t* d_id_bounds = nullptr;
    uint32_t* d_cell_bounds = nullptr;
    double* idt = nullptr;
    double* it = nullptr;
    double* irec = nullptr;
    uint32_t* pcount = nullptr;
    std::vector<sph_scheme> batch_schemes;
    std::vector<double> batch_dt;

    // captured step graphs, one per parity of `cur`
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    bool graph_timed = false;
    // persistent step form: the one cooperative launch of a step captured per parity of
    // `cur` (null: not captured yet; fused_direct: the runtime refused the capture, the
    // launches go straight to the stream)
    cudaGraphExec_t fgraph[2] = {nullptr, nullptr};
    bool fused_direct = false;
    std::vector<unsigned char> tab_host;  // copy of the device instance table
};

namespace {

sph_status fail(sph_ctx* c, sph_status s, const std::string& msg) {
    if (c) c->err = msg;
    else g_create_error = msg;
    return s;
}

sph_status cuda_fail(sph_ctx* c, cudaError_t e, const char* what) {
    return fail(c, SPH_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                              \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, #call); \
    } while (0)

double support_factor(int kernel) { return kernel == SPH_KERNEL_QUINTIC ? 3.0 : 2.0; }

// Normalisation of the unscaled smoothing functions of sph_device.cuh (the cubic spline
// there is four times the M4 B-spline, whose factors are 10 / (7 pi) and 1 / pi).
double sigma(int kernel, int dim) {
    if (kernel == SPH_KERNEL_QUINTIC) return dim == 2 ? 7.0 / (478.0 * PI) : 1.0 / (120.0 * PI);
    if (kernel == SPH_KERNEL_CUBIC_SPLINE) return dim == 2 ? 5.0 / (14.0 * PI) : 1.0 / (4.0 * PI);
    return dim == 2 ? 7.0 / (4.0 * PI) : 21.0 / (16.0 * PI);
}

// Cells no smaller than the support radius (with a 1e-5 relative margin so that the
// mode-precision neighbour test never accepts a pair two cells apart).
sph_status make_grid(sph_ctx* c, const sph_domain& D, Grid* G) {
    if (D.dim != 2 && D.dim != 3) return fail(c, SPH_ERR_INVALID, "dim must be 2 or 3");
    if (D.kernel != SPH_KERNEL_QUINTIC && D.kernel != SPH_KERNEL_WENDLAND_C2 &&
        D.kernel != SPH_KERNEL_CUBIC_SPLINE)
        return fail(c, SPH_ERR_INVALID, "unknown kernel");
    if (D.precision != SPH_PREC_FP64 && D.precision != SPH_PREC_FP32)
        return fail(c, SPH_ERR_INVALID, "unknown precision");
    const double kh = support_factor(D.kernel) * D.h;
    if (!(D.h > 0.0) || !std::isfinite(kh)) return fail(c, SPH_ERR_INVALID, "h must be > 0");
    // cells of side >= kh / R (R = 1 in 2D, 2 in 3D: the stencil of stencil.cuh)
    const int R = D.dim == 3 ? 2 : 1;
    G->dim = D.dim;
    double ncells = 1.0;
    for (int d = 0; d < 3; ++d) {
        if (d < D.dim) {
            const double ext = D.hi[d] - D.lo[d];
            if (!(ext > 0.0)) return fail(c, SPH_ERR_INVALID, "empty cell box");
            double nd = std::floor(ext / (kh / R * 1.00001));
            if (nd < 1.0) nd = 1.0;
            if (nd > 1e7) return fail(c, SPH_ERR_INVALID, "too many cells");
            G->nc[d] = (int)nd;
            G->periodic[d] = D.periodic[d] ? 1 : 0;
            if (G->periodic[d] && G->nc[d] < 2 * R + 1)
                return fail(c, SPH_ERR_INVALID, "a periodic axis needs at least 2R + 1 cells (3 in 2D, 5 in 3D)");
            G->cs[d] = ext / (double)G->nc[d];
            G->lo_f[d] = (float)D.lo[d];
            G->inv_cs_f[d] = (float)(1.0 / G->cs[d]);
            G->lo[d] = D.lo[d];
            G->hi[d] = D.hi[d];
            G->L[d] = ext;
        } else {
            G->nc[d] = 1;
            G->periodic[d] = 0;
            G->cs[d] = 1.0;
            G->lo_f[d] = 0.0f;
            G->inv_cs_f[d] = 1.0f;
            G->lo[d] = 0.0;
            G->hi[d] = 1.0;
            G->L[d] = 1.0;
        }
        ncells *= G->nc[d];
    }
    if (ncells > 2147483000.0) return fail(c, SPH_ERR_INVALID, "too many cells");
    G->ncells = (int)ncells;
    // With >= 2R + 3 cells on every periodic axis a source run of the stencil either lies
    // within R + 1 cells (|dx| <= (R + 1) L / (2R + 3) < L / 2: the minimum image never
    // applies) or wraps around the box (|dx| > L - (R + 1) cs > L / 2: it always applies,
    // with the sign of the wrap), so the pair loops can apply it per run with the same
    // arithmetic.
    G->run_shift = 1;
    for (int d = 0; d < D.dim; ++d)
        if (G->periodic[d] && G->nc[d] < 2 * R + 3) G->run_shift = 0;
    return SPH_OK;
}

template <class Real>
PairConst<Real> pair_const_dg(const sph_domain& D, const Grid& Gr, const sph_scheme* s) {
    PairConst<Real> K{};
    for (int d = 0; d < 3; ++d) {
        K.L[d] = (Real)(Gr.L[d]);
        K.halfL[d] = K.L[d] * (Real)0.5;
    }
    const Real kh = (Real)support_factor(D.kernel) * (Real)D.h;
    K.kh2 = kh * kh;
    K.h = (Real)D.h;
    K.inv_h = (Real)(1.0 / D.h);
    const double sg = sigma(D.kernel, D.dim);
    const double hd = std::pow(D.h, D.dim);
    K.wfac = (Real)(sg / hd);
    K.gfac = (Real)(sg / (hd * D.h * D.h));
    if (s) {
        K.eta_h2 = (Real)(s->eta * D.h * D.h);
        K.av_h2 = (Real)(0.01 * D.h * D.h);
        K.nu4 = (Real)(4.0 * s->nu);
        K.alpha_c0 = (Real)(s->alpha * s->c0);
        K.c0 = (Real)s->c0;
        K.xsph = (Real)s->xsph_eps;
        int f = 0;
        if (s->density == SPH_DENSITY_CONTINUITY) f |= F_CONTINUITY;
        if (s->nu != 0.0) f |= F_LAMINAR;
        if (s->alpha != 0.0) f |= F_AV;
        if (s->xsph_eps != 0.0) f |= F_XSPH;
        if (s->wall_bc == SPH_WALL_ADAMI) f |= F_WALLP;
        if (s->density == SPH_DENSITY_EDAC) {
            f |= F_EDAC;
            K.inv_rho0 = (Real)(1.0 / s->rho0);
            K.edac_d = (Real)(2.0 * (D.h * s->c0 / 16.0) / s->rho0);  // 2 nu_e / rho0
            K.c02 = (Real)(s->c0 * s->c0);
        }
        K.flags = f;
    }
    return K;
}

template <class Real>
PairConst<Real> pair_const(const sph_ctx* c, const sph_scheme* s) {
    return pair_const_dg<Real>(c->dom, c->G, s);
}

StepConst step_const_d(const sph_domain& D, const sph_scheme* s, double dt_fixed) {
    StepConst C{};
    C.rho0 = s->rho0;
    C.inv_rho0 = 1.0 / s->rho0;
    C.gamma = s->gamma;
    C.B = s->c0 * s->c0 * s->rho0 / s->gamma;
    for (int d = 0; d < 3; ++d) C.g[d] = s->g[d];
    C.h = D.h;
    C.c0 = s->c0;
    C.nu = s->nu;
    C.dt_fixed = dt_fixed;
    C.continuity = s->density == SPH_DENSITY_CONTINUITY;
    C.gamma7 = s->gamma == 7.0;
    C.precision = D.precision;
    return C;
}

StepConst step_const(const sph_ctx* c, const sph_scheme* s, double dt_fixed) {
    return step_const_d(c->dom, s, dt_fixed);
}

sph_status check_scheme(sph_ctx* c, const sph_scheme* s) {
    if (!s) return fail(c, SPH_ERR_INVALID, "scheme is NULL");
    if (s->density != SPH_DENSITY_CONTINUITY && s->density != SPH_DENSITY_SUMMATION &&
        s->density != SPH_DENSITY_EDAC)
        return fail(c, SPH_ERR_INVALID, "unknown density formulation");
    if (s->density == SPH_DENSITY_EDAC && c && c->nwall > 0)
        return fail(c, SPH_ERR_INVALID, "the EDAC form is built for fluid-only problems");
    if (s->density == SPH_DENSITY_EDAC && s->integrator != SPH_INTEGRATOR_KDK)
        return fail(c, SPH_ERR_INVALID, "the EDAC form runs with the kick-drift-kick integrator");
    if (!(s->rho0 > 0.0) || !(s->c0 > 0.0) || !(s->gamma > 0.0))
        return fail(c, SPH_ERR_INVALID, "rho0, c0 and gamma must be > 0");
    if (!(s->nu >= 0.0) || !(s->eta >= 0.0) || !(s->alpha >= 0.0) || !std::isfinite(s->xsph_eps))
        return fail(c, SPH_ERR_INVALID, "nu, eta, alpha must be >= 0");
    if (s->wall_bc != SPH_WALL_DENSITY && s->wall_bc != SPH_WALL_ADAMI)
        return fail(c, SPH_ERR_INVALID, "unknown wall condition");
    if (s->integrator != SPH_INTEGRATOR_KDK && s->integrator != SPH_INTEGRATOR_PEC)
        return fail(c, SPH_ERR_INVALID, "unknown integrator");
    if (s->reserved != 0) return fail(c, SPH_ERR_INVALID, "scheme.reserved must be 0");
    return SPH_OK;
}

bool same_scheme(const sph_scheme& a, const sph_scheme& b) { return std::memcmp(&a, &b, sizeof a) == 0; }

// Neighbour build: [drift] + keys, radix sort, gather into the other set (+EOS shadow),
// cell table. Enqueued on the context stream (capturable).
int tindex(int T) { return T == 1 ? 0 : (T == 2 ? 1 : (T == 4 ? 2 : 3)); }

// Grid of a pair pass: one group of T lanes per particle, capped at what fits on the GPU.
int pass_grid(const sph_ctx* c, int pass, int T) {
    long long want = ((long long)c->N * T + pair_threads() - 1) / pair_threads();
    long long cap = (long long)c->sms * c->bps[pass][tindex(T)];
    long long g = want < cap ? want : cap;
    return g < 1 ? 1 : (int)g;
}

void set_groups(sph_ctx* c, int td, int tm) {
    c->group_d = td;
    c->group_m = tm;
    c->grid_d = pass_grid(c, 0, td);
    c->grid_m = pass_grid(c, 1, tm);
}

// Process-wide autotuner cache: (precision, dim, kernel, log2 N) -> group sizes.
struct TuneKey {
    int precision, dim, kernel, nbucket;
    bool operator==(const TuneKey& o) const {
        return precision == o.precision && dim == o.dim && kernel == o.kernel && nbucket == o.nbucket;
    }
};
std::mutex g_tune_lock;
struct TuneVal {
    int lanes;   // momentum-pass lanes per destination
    int mode;    // SPH_STEP_GRAPH or SPH_STEP_PERSISTENT
    int dlanes;  // density-pass lanes per destination
};
std::vector<std::pair<TuneKey, TuneVal>> g_tune_cache;

TuneKey tune_key(const sph_ctx* c) {
    int b = 0;
    while ((1ll << (b + 1)) <= (long long)c->N) ++b;
    return TuneKey{c->dom.precision, c->dom.dim, c->dom.kernel, b};
}

// Tuning before any autotune call: a cached result for this shape, else 4 momentum lanes
// below 200,000 particles and 1 above, and the per-phase graph.
void default_tuning(const sph_ctx* c, int* td, int* tm, int* mode) {
    *mode = SPH_STEP_GRAPH;
    {
        std::lock_guard<std::mutex> lock(g_tune_lock);
        const TuneKey k = tune_key(c);
        for (auto& e : g_tune_cache)
            if (e.first == k) {
                *tm = e.second.lanes;
                *td = e.second.dlanes;
                *mode = e.second.mode;
                return;
            }
    }
    *tm = c->N < 200000 ? 4 : 1;
    *td = *tm;
}

void remember_tuning(const sph_ctx* c) {
    std::lock_guard<std::mutex> lock(g_tune_lock);
    const TuneKey k = tune_key(c);
    const TuneVal v{c->group_m, c->step_mode, c->group_d};
    for (auto& e : g_tune_cache)
        if (e.first == k) {
            e.second = v;
            return;
        }
    g_tune_cache.push_back({k, v});
}

void mark(sph_ctx* c, int k, bool timed) {
    if (timed) cudaEventRecordWithFlags(c->ev[k], c->stream, cudaEventRecordExternal);
}

int ntab(const sph_ctx* c) { return c->ninst ? c->ninst : 1; }

// Launch description of the context's current state (instance table, buffers).
StepLaunch step_launch(sph_ctx* c, int kick) {
    StepLaunch L{};
    L.precision = c->dom.precision;
    L.dim = c->dom.dim;
    L.kernel = c->dom.kernel;
    L.n = c->N;
    L.sms = c->sms;
    L.ninst = ntab(c);
    L.kick = kick;
    L.maxn = c->maxn;
    L.group_d = c->group_d;
    L.group_m = c->group_m;
    L.grid_d = c->grid_d;
    L.grid_m = c->grid_m;
    L.finalize = c->ninst == 0;
    L.tab = c->d_tab;
    L.tab_host = (c->ninst == 0 && !c->tab_host.empty()) ? (const void*)c->tab_host.data() : nullptr;
    L.id_bounds = c->d_id_bounds;
    L.cell_bounds = c->d_cell_bounds;
    L.idt = c->ninst ? c->idt : &c->ctl->dt;
    L.it = c->it;
    L.irec = c->irec;
    L.Sin = c->set[c->cur];
    L.S = c->set[c->cur];
    L.P = c->P;
    L.Q = c->Q;
    L.R = c->R;
    L.E = c->E;
    L.edac = c->edac ? 1 : 0;
    L.skeys = c->skeys;
    L.off = c->off;
    L.cpart = c->ninst == 0 ? c->cpart : nullptr;
    L.dyn = (c->ninst == 0 ? 1 : 0) | (c->nwall > 0 ? 2 : 0);
    L.nl = c->nl;
    L.cnt = c->cnt;
    L.pcount = c->pcount;
    L.bpart = c->bpart;
    L.pm = c->pm;
    L.pd = c->pd;
    L.history = c->history;
    L.ctl = c->ctl;
    return L;
}

// Neighbour build: [drift] + keys, radix sort, gather into the other set (+EOS shadow),
// cell table. Enqueued on the context stream (capturable); constants from the table.
// The sort workspace is zero after every completed build (the reorder kernel clears it);
// it is cleared on the stream only when a build may have stopped part-way. Called before
// graph capture and before graph launches, so captured steps hold no memset of it.
cudaError_t clear_work_if_dirty(sph_ctx* c) {
    if (!c->work_dirty) return cudaSuccess;
    c->work_dirty = false;
    return cudaMemsetAsync(c->sort_work, 0, sort_work_words(c->N, c->passes) * 4, c->stream);
}

void enqueue_build(sph_ctx* c, int drift, int kick, int carry_rates, bool timed = false) {
    cudaStream_t st = c->stream;
    clear_work_if_dirty(c);
    cudaMemsetAsync(&c->ctl->outside, 0, sizeof(unsigned), st);
    StepLaunch L = step_launch(c, kick);
    mark(c, 0, timed);
    launch_keys_hist(L, drift, c->keys[0], c->passes, c->sort_work, st);
    mark(c, 1, timed);
    const int b = launch_onesweep(c->N, c->keys, c->vals, c->passes, c->sort_work, c->ctl, c->wait_ns, st);
    c->skeys = c->keys[b];
    c->perm = c->vals[b];
    mark(c, 2, timed);
    const int nxt = c->cur ^ 1;
    L.S = c->set[nxt];
    L.skeys = c->skeys;
    launch_reorder(L, c->vals[b], carry_rates, c->off, c->G.ncells, c->sort_work,
                   (int)sort_work_words(c->N, c->passes), st);
    mark(c, 3, timed);  // the cell table is written by the reorder kernel
    mark(c, 4, timed);
    c->cur = nxt;
}

// Density pass, then momentum pass (+ the per-instance reduction of a batch).
void enqueue_eval(sph_ctx* c, int kick, bool timed = false) {
    const StepLaunch L = step_launch(c, kick);
    launch_density_pass(L, c->stream);
    if (c->wall_pass) launch_wall_pressure(L, c->stream);
    mark(c, 5, timed);
    launch_momentum_pass(L, c->stream);
    if (!L.finalize) launch_batch_reduce(L, c->stream);
}

// ------------------------------------------------------------ persistent step
constexpr int FUSED_MAX_BPS = 8;

// Grid of the persistent kernel: enough blocks for one group of T lanes per particle,
// capped at the blocks that are co-resident (a cooperative launch needs all of them).
int fused_grid(const sph_ctx* c) {
    int bps = c->fused_bps[tindex(c->group_m)];
    if (bps > FUSED_MAX_BPS) bps = FUSED_MAX_BPS;
    const long long cap = (long long)c->sms * bps;
    const long long want = ((long long)c->N * c->group_m + FUSED_THREADS - 1) / FUSED_THREADS;
    long long g = want < cap ? want : cap;
    return g < 1 ? 1 : (int)g;
}

FusedLaunch fused_launch(sph_ctx* c) {
    FusedLaunch F{};
    F.L = step_launch(c, 1);
    F.L.Sin = c->set[c->cur];
    F.L.S = c->set[c->cur ^ 1];
    for (int k = 0; k < 2; ++k) {
        F.keys[k] = c->keys[k];
        F.vals[k] = c->vals[k];
    }
    F.work = c->sort_work;
    F.work_words = (int)sort_work_words(c->N, c->passes);
    F.off = c->off;
    F.part = c->fpart;
    F.passes = c->passes;
    F.ntiles = onesweep_tiles(c->N);
    F.ncells = c->G.ncells;
    F.wall_pass = c->wall_pass ? 1 : 0;
    F.wait_ns = c->wait_ns;
    return F;
}

// Captures the persistent step (its one cooperative launch) once per parity of the set in
// use. The kernel leaves the barrier words, the sort workspace and the clamp counter as it
// found them, so a graph holds the launch alone; the limits of its waits and its grid are
// baked in (set_groups and sph_set_wait_limit drop the graphs). Returns false, with no
// graph kept, where the runtime does not capture a cooperative launch.
bool capture_fused_graphs(sph_ctx* c, int grid) {
    const int cur0 = c->cur;
    bool ok = true;
    for (int k = 0; k < 2 && ok; ++k) {
        c->cur = cur0 ^ k;
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            ok = false;
            break;
        }
        const FusedLaunch F = fused_launch(c);
        const cudaError_t le = launch_fused(F, c->group_m, grid, c->stream);
        const cudaError_t ee = cudaStreamEndCapture(c->stream, &g);
        cudaGraphExec_t ex = nullptr;
        if (le != cudaSuccess || ee != cudaSuccess || !g || cudaGraphInstantiate(&ex, g, 0) != cudaSuccess)
            ok = false;
        if (g) cudaGraphDestroy(g);
        if (ok) c->fgraph[cur0 ^ k] = ex;
    }
    c->cur = cur0;
    if (!ok) {
        cudaGetLastError();
        for (int k = 0; k < 2; ++k)
            if (c->fgraph[k]) {
                cudaGraphExecDestroy(c->fgraph[k]);
                c->fgraph[k] = nullptr;
            }
    }
    return ok;
}

// nsteps persistent steps (one cooperative launch each, replayed from the captured step
// graph of the current parity) on the context stream.
sph_status run_fused(sph_ctx* c, int nsteps) {
    if (c->fused_bps[tindex(c->group_m)] < 1)
        return fail(c, SPH_ERR_INVALID, "the persistent step kernel cannot be resident on this device");
    CK(cudaMemsetAsync(&c->ctl->outside, 0, sizeof(unsigned), c->stream));
    CK(cudaMemsetAsync(&c->ctl->bar_count, 0, sizeof(unsigned), c->stream));
    CK(cudaMemsetAsync(&c->ctl->bar_gen, 0, sizeof(unsigned), c->stream));
    CK(cudaMemsetAsync(c->sort_work, 0, sort_work_words(c->N, c->passes) * 4, c->stream));
    const int grid = fused_grid(c);
    if (!c->fgraph[0] && !c->fused_direct) c->fused_direct = !capture_fused_graphs(c, grid);
    for (int k = 0; k < nsteps; ++k) {
        if (c->fgraph[c->cur]) {
            CK(cudaGraphLaunch(c->fgraph[c->cur], c->stream));
        } else {
            const FusedLaunch F = fused_launch(c);
            const cudaError_t e = launch_fused(F, c->group_m, grid, c->stream);
            if (e != cudaSuccess) return cuda_fail(c, e, "persistent step launch");
        }
        c->cur ^= 1;
    }
    c->skeys = c->keys[c->passes & 1];
    c->last_fused = true;
    return SPH_OK;
}

sph_status capture_step_graphs(sph_ctx* c);

// One step of the midpoint integrator (rates at the current state valid): predictor in
// place, build + evaluation at the midpoint, corrector on the midpoint order, build +
// evaluation at the end of the step (the timed phases), record. Two builds: the set in
// use is the same at the end.
void enqueue_pec_step(sph_ctx* c) {
    const int cont = c->pec_cont;
    const int dim = c->dom.dim;
    const int prec = c->dom.precision;
    double* dt_step = c->pec_save + (size_t)(2 * dim + 1) * c->N;
    if (c->ninst)
        launch_pec_predict_batch(c->set[c->cur], c->pec_save, c->N, dim, prec, c->d_tab,
                                 c->d_cell_bounds, c->ninst, c->skeys, c->idt, dt_step, cont,
                                 c->ctl, c->sms, c->stream);
    else
        launch_pec_predict(c->set[c->cur], c->pec_save, c->N, dim, c->G, &c->ctl->dt, dt_step,
                           cont, c->ctl, c->sms, c->stream);
    enqueue_build(c, 0, 0, 0);
    enqueue_eval(c, 0);
    if (c->ninst)
        launch_pec_correct_batch(c->set[c->cur], c->pec_save, c->perm, c->N, dim, prec, c->d_tab,
                                 c->d_cell_bounds, c->ninst, c->skeys, dt_step, cont, c->ctl,
                                 c->sms, c->stream);
    else
        launch_pec_correct(c->set[c->cur], c->pec_save, c->perm, c->N, dim, c->G, dt_step, cont,
                           c->ctl, c->sms, c->stream);
    enqueue_build(c, 0, 0, 0, c->timing);
    enqueue_eval(c, 0, c->timing);
    if (c->ninst) launch_pec_record_batch(c->it, c->irec, dt_step, c->ninst, c->ctl, c->stream);
    else launch_pec_record(c->ctl, c->history, dt_step, c->stream);
}

// nsteps steps in the context's mode (tables already uploaded, rates valid).
sph_status run_steps(sph_ctx* c, int nsteps) {
    if (nsteps <= 0) return SPH_OK;
    // the persistent kernel runs one evaluation per step: midpoint steps run as the graph
    if (c->step_mode == SPH_STEP_PERSISTENT && !c->pec) return run_fused(c, nsteps);
    if (!c->graph[0] || c->graph_timed != c->timing) {
        sph_status s = capture_step_graphs(c);
        if (s != SPH_OK) return s;
    }
    CK(clear_work_if_dirty(c));
    for (int k = 0; k < nsteps; ++k) {
        CK(cudaGraphLaunch(c->graph[c->cur], c->stream));
        if (!c->pec) c->cur ^= 1;  // one build per step, or two
    }
    c->skeys = c->keys[c->passes & 1];
    c->last_fused = false;
    return SPH_OK;
}

// Instance table on the device: one entry (a single problem: its domain, scheme, dt) or
// one per batch instance. Uploaded outside graph capture when it changes.
template <class Real>
void table_bytes(const sph_ctx* c, const sph_scheme* schemes, const double* dts,
                 std::vector<unsigned char>& bytes) {
    const int nt = ntab(c);
    bytes.assign((size_t)nt * sizeof(Inst<Real>), 0);
    Inst<Real>* T = (Inst<Real>*)bytes.data();
    for (int k = 0; k < nt; ++k) {
        const sph_domain& D = c->ninst ? c->doms[k] : c->dom;
        const Grid& Gk = c->ninst ? c->grids[k] : c->G;
        Inst<Real> I{};
        I.G = Gk;
        I.K = pair_const_dg<Real>(D, Gk, &schemes[k]);
        I.C = step_const_d(D, &schemes[k], dts[k] > 0.0 ? dts[k] : 0.0);
        I.cell_base = c->ninst ? c->cell_bounds_h[k] : 0u;
        I.cell_base_end = c->ninst ? c->cell_bounds_h[k + 1] : (uint32_t)c->G.ncells;
        T[k] = I;
    }
}

void drop_graphs(sph_ctx* c);

sph_status upload_table(sph_ctx* c, const sph_scheme* schemes, const double* dts) {
    bool wp = false;
    for (int k = 0; k < ntab(c); ++k) wp |= schemes[k].wall_bc == SPH_WALL_ADAMI;
    wp &= c->nwall > 0;
    if (wp != c->wall_pass) {  // the captured steps hold the pass or not
        c->wall_pass = wp;
        drop_graphs(c);
    }
    const bool pec = schemes[0].integrator == SPH_INTEGRATOR_PEC;  // shared by a batch
    if (pec && !c->pec_save) {  // outside any capture: the first use of the integrator
        const size_t bytes = ((size_t)(2 * c->dom.dim + 1) * c->N + ntab(c)) * sizeof(double);
        void* p = nullptr;
        if (c->alloc) p = c->alloc(bytes, c->user);
        else if (cudaMalloc(&p, bytes) != cudaSuccess) p = nullptr;
        if (!p) {
            cudaGetLastError();
            return fail(c, SPH_ERR_OOM, "midpoint integrator state of " + std::to_string(bytes) + " bytes");
        }
        c->pec_save = (double*)p;
    }
    const bool edac = schemes[0].density == SPH_DENSITY_EDAC;  // shared by a batch
    if (edac != c->edac) {  // the captured reorder gathers the pressure or not
        c->edac = edac;
        drop_graphs(c);
    }
    const int cont = schemes[0].density != SPH_DENSITY_SUMMATION;
    if (pec != c->pec || (pec && cont != c->pec_cont)) {  // captured steps: one integrator
        c->pec = pec;
        c->pec_cont = cont;
        drop_graphs(c);
    }
    std::vector<unsigned char> bytes;
    if (c->dom.precision) table_bytes<float>(c, schemes, dts, bytes);
    else table_bytes<double>(c, schemes, dts, bytes);
    if (bytes == c->tab_host) return SPH_OK;
    CK(cudaMemcpyAsync(c->d_tab, bytes.data(), bytes.size(), cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->tab_host.swap(bytes);
    // the pair passes of a single problem take the entry by value: captured steps hold it
    if (c->ninst == 0) drop_graphs(c);
    return SPH_OK;
}

sph_status upload_single(sph_ctx* c, const sph_scheme* s, double dt_fixed) {
    return upload_table(c, s, &dt_fixed);
}

sph_status sync_status(sph_ctx* c) {
    unsigned status = 0;
    CK(cudaMemcpyAsync(&status, &c->ctl->status, sizeof status, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    CK(cudaGetLastError());
    if (status) c->work_dirty = true;
    if (status & ST_NONFINITE) return fail(c, SPH_ERR_NONFINITE, "non-finite state detected");
    if (status & ST_TIMEOUT) return fail(c, SPH_ERR_TIMEOUT, "device wait timed out");
    if (status & ST_CAPACITY)
        return fail(c, SPH_ERR_CAPACITY,
                    "a particle has more neighbours than the list capacity (" +
                        std::to_string(c->maxn) + "); set the state again to re-size it");
    return SPH_OK;
}

void drop_graphs(sph_ctx* c) {
    for (int k = 0; k < 2; ++k) {
        if (c->graph[k]) {
            cudaGraphExecDestroy(c->graph[k]);
            c->graph[k] = nullptr;
        }
        if (c->fgraph[k]) {
            cudaGraphExecDestroy(c->fgraph[k]);
            c->fgraph[k] = nullptr;
        }
    }
}

void free_dev(sph_ctx* c, void* p) {
    if (!p) return;
    if (c->free_fn) c->free_fn(p, c->user);
    else cudaFree(p);
}

// Neighbour-list capacity: count the neighbours of every particle at the current cell
// table and make room for twice the largest count (+32), rounded up to a multiple of 32.
sph_status ensure_list_capacity(sph_ctx* c) {
    const PairConst<float> Kf = pair_const<float>(c, nullptr);
    const PairConst<double> Kd = pair_const<double>(c, nullptr);
    uint32_t* d_counts = (uint32_t*)c->io;
    launch_export_neighbors(c->dom.precision, c->dom.dim, c->P, c->skeys, c->off,
                            c->set[c->cur].tag, c->N, c->G, Kf, Kd, 0, d_counts, nullptr, nullptr,
                            c->stream, c->sms);
    CK(cudaGetLastError());
    std::vector<uint32_t> counts(c->N);
    CK(cudaMemcpyAsync(counts.data(), d_counts, (size_t)c->N * 4, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    uint32_t mx = 0;
    for (uint32_t v : counts) mx = v > mx ? v : mx;
    if (c->nl && (uint32_t)c->maxn >= mx + mx / 4 + 8) return SPH_OK;
    int want = (int)((2 * mx + 32 + 31) / 32 * 32);
    void* p = nullptr;
    const size_t bytes = (size_t)want * c->N * 4;
    if (c->alloc) p = c->alloc(bytes, c->user);
    else if (cudaMalloc(&p, bytes) != cudaSuccess) p = nullptr;
    if (!p) {
        cudaGetLastError();
        return fail(c, SPH_ERR_OOM, "neighbour list of " + std::to_string(bytes) + " bytes");
    }
    CK(cudaStreamSynchronize(c->stream));
    free_dev(c, c->nl);
    c->nl = (uint32_t*)p;
    c->maxn = want;
    drop_graphs(c);
    return SPH_OK;
}

// Initial right-hand side at the current state (no drift, no kick).
sph_status initial_eval(sph_ctx* c, const sph_scheme* s, double dt_fixed) {
    sph_status st = upload_single(c, s, dt_fixed);
    if (st != SPH_OK) return st;
    enqueue_build(c, 0, 0, 0);
    st = ensure_list_capacity(c);
    if (st != SPH_OK) return st;
    enqueue_eval(c, 0);
    CK(cudaGetLastError());
    c->have_rates = true;
    c->nbr_valid = true;
    c->rates_scheme = *s;
    return SPH_OK;
}

// Captures one step for each parity of the set in use. The constants live in the device
// table, so the graphs stay valid when a scheme or dt changes; they are recaptured when
// the buffers, the tile shape or the timing mode change (drop_graphs).
sph_status capture_step_graphs(sph_ctx* c) {
    drop_graphs(c);
    CK(clear_work_if_dirty(c));  // outside the capture
    const int cur0 = c->cur;
    for (int k = 0; k < 2; ++k) {
        c->cur = cur0 ^ k;
        cudaGraph_t g = nullptr;
        CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
        if (c->pec) enqueue_pec_step(c);
        else {
            enqueue_build(c, 1, 1, 0, c->timing);
            enqueue_eval(c, 1, c->timing);
        }
        mark(c, 6, c->timing);
        cudaError_t e = cudaStreamEndCapture(c->stream, &g);
        if (e != cudaSuccess) {
            c->cur = cur0;
            return cuda_fail(c, e, "cudaStreamEndCapture");
        }
        cudaGraphExec_t ex = nullptr;
        e = cudaGraphInstantiate(&ex, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            c->cur = cur0;
            return cuda_fail(c, e, "cudaGraphInstantiate");
        }
        c->graph[cur0 ^ k] = ex;
    }
    c->cur = cur0;
    c->graph_timed = c->timing;
    return SPH_OK;
}

void* arena_take(char*& p, size_t bytes) {
    void* r = p;
    p += (bytes + 255) & ~size_t(255);
    return r;
}

sph_status prop_field(sph_ctx* c, const char* prop, bool writable, double** field) {
    if (!prop) return fail(c, SPH_ERR_INVALID, "prop is NULL");
    ParticleSet& S = c->set[c->cur];
    struct { const char* name; double* f; bool w; } table[] = {
        {"x", S.x[0], true}, {"y", S.x[1], true}, {"z", S.x[2], true},
        {"u", S.u[0], true}, {"v", S.u[1], true}, {"w", S.u[2], true},
        {"rho", S.rho, true}, {"m", S.m, true}, {"p", S.p, true},
        {"arho", S.arho, false}, {"ax", S.a[0], false}, {"ay", S.a[1], false}, {"az", S.a[2], false},
        {"xsx", S.xs[0], false}, {"xsy", S.xs[1], false}, {"xsz", S.xs[2], false}};
    for (auto& t : table)
        if (std::strcmp(t.name, prop) == 0) {
            if (writable && !t.w) return fail(c, SPH_ERR_INVALID, std::string("read-only property ") + prop);
            *field = t.f;
            return SPH_OK;
        }
    return fail(c, SPH_ERR_INVALID, std::string("unknown property ") + prop);
}

sph_status array_range(sph_ctx* c, int32_t array, uint32_t* first, uint32_t* count) {
    const int na = (int)c->arr_off.size() - 1;
    if (array == -1) {
        *first = 0;
        *count = (uint32_t)c->N;
        return SPH_OK;
    }
    if (array < 0 || array >= na) return fail(c, SPH_ERR_INVALID, "array index out of range");
    *first = (uint32_t)c->arr_off[array];
    *count = (uint32_t)(c->arr_off[array + 1] - c->arr_off[array]);
    return SPH_OK;
}

sph_status ensure_neighbors(sph_ctx* c) {
    if (c->nbr_valid) return SPH_OK;
    sph_scheme dummy{};
    dummy.rho0 = 1.0;
    dummy.c0 = 1.0;
    dummy.gamma = 7.0;
    sph_status st = upload_single(c, c->have_rates ? &c->rates_scheme : &dummy, 0.0);
    if (st != SPH_OK) return st;
    enqueue_build(c, 0, 0, c->have_rates ? 1 : 0);
    CK(cudaGetLastError());
    c->nbr_valid = true;
    return SPH_OK;
}

}  // namespace

namespace sph {
void set_global_error(const std::string& msg) { g_create_error = msg; }
}  // namespace sph

extern "C" void sph_destroy(sph_ctx* c);

namespace {

// Context creation for one problem (ninst = 0) or a batch of ninst instances, whose
// arrays follow each other (arrays_per_inst[k] arrays for instance k).
sph_status create_impl(const sph_domain* domains, int ninst, const sph_array_desc* arrays,
                       const int32_t* arrays_per_inst, int32_t n_arrays, void* stream,
                       sph_alloc_fn alloc, sph_free_fn free_fn, void* alloc_user, sph_ctx** out) {
    if (!out) return fail(nullptr, SPH_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (!domains || !arrays || n_arrays < 1) return fail(nullptr, SPH_ERR_INVALID, "no arrays");
    if ((alloc == nullptr) != (free_fn == nullptr))
        return fail(nullptr, SPH_ERR_INVALID, "give both allocator callbacks or neither");
    sph_ctx* c = new (std::nothrow) sph_ctx();
    if (!c) return fail(nullptr, SPH_ERR_OOM, "host allocation failed");
    const sph_domain* domain = &domains[0];
    c->dom = *domain;
    Grid G{};
    sph_status s = make_grid(c, *domain, &G);
    if (s != SPH_OK) {
        g_create_error = c->err;
        delete c;
        return s;
    }
    c->G = G;
    if (ninst > 0) {
        // per-instance grids; global cell ids are consecutive per instance
        c->ninst = ninst;
        c->doms.assign(domains, domains + ninst);
        c->grids.resize(ninst);
        c->cell_bounds_h.assign(1, 0);
        double total = 0.0;
        int na = 0;
        for (int k = 0; k < ninst; ++k) {
            const sph_domain& D = domains[k];
            if (D.dim != domain->dim || D.kernel != domain->kernel || D.precision != domain->precision) {
                g_create_error = "batch instances must share dim, kernel and precision";
                delete c;
                return SPH_ERR_INVALID;
            }
            s = make_grid(c, D, &c->grids[k]);
            if (s != SPH_OK) {
                g_create_error = "instance " + std::to_string(k) + ": " + c->err;
                delete c;
                return s;
            }
            total += c->grids[k].ncells;
            if (total > 2147483000.0) {
                g_create_error = "too many cells in the batch";
                delete c;
                return SPH_ERR_INVALID;
            }
            c->cell_bounds_h.push_back((uint32_t)total);
            if (!arrays_per_inst || arrays_per_inst[k] < 1) {
                g_create_error = "every instance needs at least one array";
                delete c;
                return SPH_ERR_INVALID;
            }
            na += arrays_per_inst[k];
        }
        if (na != n_arrays) {
            g_create_error = "arrays_per_instance does not add up to the array count";
            delete c;
            return SPH_ERR_INVALID;
        }
        c->G.ncells = (int)total;
    }
    c->arr_off.assign(1, 0);
    for (int a = 0; a < n_arrays; ++a) {
        const sph_array_desc& A = arrays[a];
        if (A.n < 0 || (A.n > 0 && (!A.x || !A.y || !A.rho || !A.m)) ||
            (domain->dim == 3 && A.n > 0 && !A.z) ||
            (A.role != SPH_ROLE_FLUID && A.role != SPH_ROLE_WALL)) {
            g_create_error = "array " + std::to_string(a) + ": missing x, y, (z), rho or m, or bad role";
            delete c;
            return SPH_ERR_INVALID;
        }
        c->arr_off.push_back(c->arr_off.back() + A.n);
    }
    if (c->arr_off.back() > 0x3ffffff0LL || c->arr_off.back() < 1) {
        g_create_error = "particle count must be in [1, 2^30)";
        delete c;
        return SPH_ERR_INVALID;
    }
    c->N = (int)c->arr_off.back();
    if (ninst > 0) {
        c->id_bounds_h.assign(1, 0);
        int a = 0;
        for (int k = 0; k < ninst; ++k) {
            a += arrays_per_inst[k];
            c->id_bounds_h.push_back((uint32_t)c->arr_off[a]);
        }
    } else {  // a single problem is a table of one instance
        c->id_bounds_h = {0u, (uint32_t)c->N};
        c->cell_bounds_h = {0u, (uint32_t)c->G.ncells};
    }
    c->alloc = alloc;
    c->free_fn = free_fn;
    c->user = alloc_user;

    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->device);
    if (e != cudaSuccess) {
        g_create_error = std::string("no CUDA device: ") + cudaGetErrorString(e);
        delete c;
        return SPH_ERR_CUDA;
    }
    if (stream) {
        c->stream = (cudaStream_t)stream;
    } else {
        e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            g_create_error = std::string("cudaStreamCreate: ") + cudaGetErrorString(e);
            delete c;
            return SPH_ERR_CUDA;
        }
        c->own_stream = true;
    }
    c->passes = radix_passes(c->G.ncells);  // global cell ids of all instances
    if (c->passes < 1) c->passes = 1;
    c->grid_cap = 1;
    for (int pass = 0; pass < 2; ++pass)
        for (int k = 0; k < 4; ++k) {
            c->bps[pass][k] = pairs_max_blocks_per_sm(domain->precision, pass, domain->dim,
                                                      domain->kernel, 1 << k, c->ninst == 0);
            if (c->sms * c->bps[pass][k] > c->grid_cap) c->grid_cap = c->sms * c->bps[pass][k];
        }
    for (int k = 0; k < 4; ++k)
        c->fused_bps[k] = fused_max_blocks_per_sm(domain->precision, domain->dim, domain->kernel, 1 << k);
    {
        int td = 1, tm = 1, mode = SPH_STEP_GRAPH;
        default_tuning(c, &td, &tm, &mode);
        set_groups(c, td, tm);
        c->step_mode = mode;
    }

    // ---- arena
    const size_t N = (size_t)c->N;
    const size_t real = domain->precision == SPH_PREC_FP32 ? 4 : 8;
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    size_t bytes = 0;
    bytes += 2 * (STATE_FIELDS * al(N * 8) + al(N * 4));       // two particle sets
    bytes += 2 * al(N * 4 * real) + al(N * real);              // shadow P, Q, R
    if (domain->precision == SPH_PREC_FP32) bytes += al(N * 16);  // position residuals E
    bytes += 4 * al(N * 4);                                    // keys, vals
    bytes += al(((size_t)c->G.ncells + 1) * 4);                // cell offsets
    bytes += al(radix_hist_words(c->N) * 4);                   // radix histograms
    bytes += al(sort_work_words(c->N, c->passes) * 4);          // one-sweep workspace
    bytes += al((size_t)c->grid_cap * 8 * 8) + al((size_t)c->grid_cap * 4 * 8);  // partials
    bytes += al(((size_t)c->N + 31) / 32 * 8 * 8);  // momentum chunk partials
    bytes += al(N * 4);                                        // neighbour-list lengths
    bytes += al((size_t)c->sms * FUSED_MAX_BPS * FUSED_PART * 8);  // persistent partials
    bytes += al(sizeof(Control));
    bytes += al((size_t)HIST_CAP * DIAG_N * 8);                // history ring
    const size_t io_bytes = al(N * 4) + 2 * al(N * 8 + 8);     // io scratch
    bytes += io_bytes;
    const size_t inst_bytes = domain->precision == SPH_PREC_FP32 ? sizeof(Inst<float>) : sizeof(Inst<double>);
    const size_t nt = ninst > 0 ? (size_t)ninst : 1;
    bytes += al(nt * inst_bytes) + 2 * al((nt + 1) * 4);        // instance table, bounds
    if (ninst > 0) bytes += 2 * al(nt * 8) + al(nt * DIAG_N * 8) + al(N * 8) + al(nt * BATCH_SPLIT * 10 * 8);
    c->arena_bytes = bytes;
    if (alloc) c->arena = alloc(bytes, alloc_user);
    else if (cudaMalloc(&c->arena, bytes) != cudaSuccess) c->arena = nullptr;
    if (!c->arena) {
        cudaGetLastError();
        g_create_error = "device allocation of " + std::to_string(bytes) + " bytes failed";
        if (c->own_stream) cudaStreamDestroy(c->stream);
        delete c;
        return SPH_ERR_OOM;
    }
    char* p = (char*)c->arena;
    for (int k = 0; k < 2; ++k) {
        ParticleSet& S = c->set[k];
        for (int d = 0; d < 3; ++d) S.x[d] = (double*)arena_take(p, N * 8);
        for (int d = 0; d < 3; ++d) S.u[d] = (double*)arena_take(p, N * 8);
        S.rho = (double*)arena_take(p, N * 8);
        S.m = (double*)arena_take(p, N * 8);
        S.arho = (double*)arena_take(p, N * 8);
        for (int d = 0; d < 3; ++d) S.a[d] = (double*)arena_take(p, N * 8);
        for (int d = 0; d < 3; ++d) S.xs[d] = (double*)arena_take(p, N * 8);
        S.p = (double*)arena_take(p, N * 8);
        S.tag = (uint32_t*)arena_take(p, N * 4);
    }
    c->P = arena_take(p, N * 4 * real);
    c->Q = arena_take(p, N * 4 * real);
    c->R = arena_take(p, N * real);
    if (domain->precision == SPH_PREC_FP32) c->E = arena_take(p, N * 16);
    for (int k = 0; k < 2; ++k) c->keys[k] = (uint32_t*)arena_take(p, N * 4);
    for (int k = 0; k < 2; ++k) c->vals[k] = (uint32_t*)arena_take(p, N * 4);
    c->off = (uint32_t*)arena_take(p, ((size_t)c->G.ncells + 1) * 4);
    c->hist = (uint32_t*)arena_take(p, radix_hist_words(c->N) * 4);
    c->sort_work = (uint32_t*)arena_take(p, sort_work_words(c->N, c->passes) * 4);
    c->pm = (double*)arena_take(p, (size_t)c->grid_cap * 8 * 8);
    c->pd = (double*)arena_take(p, (size_t)c->grid_cap * 4 * 8);
    c->cpart = (double*)arena_take(p, ((size_t)c->N + 31) / 32 * 8 * 8);
    c->cnt = (uint32_t*)arena_take(p, N * 4);
    c->fpart = (double*)arena_take(p, (size_t)c->sms * FUSED_MAX_BPS * FUSED_PART * 8);
    c->ctl = (Control*)arena_take(p, sizeof(Control));
    c->history = (double*)arena_take(p, (size_t)HIST_CAP * DIAG_N * 8);
    c->io = arena_take(p, io_bytes);
    c->skeys = c->keys[0];
    c->d_tab = arena_take(p, nt * inst_bytes);
    c->d_id_bounds = (uint32_t*)arena_take(p, (nt + 1) * 4);
    c->d_cell_bounds = (uint32_t*)arena_take(p, (nt + 1) * 4);
    if (ninst > 0) {
        c->idt = (double*)arena_take(p, (size_t)ninst * 8);
        c->it = (double*)arena_take(p, (size_t)ninst * 8);
        c->irec = (double*)arena_take(p, (size_t)ninst * DIAG_N * 8);
        c->pcount = (uint32_t*)arena_take(p, N * 8);
        c->bpart = (double*)arena_take(p, nt * BATCH_SPLIT * 10 * 8);
    }

    // ---- upload
    sph_status rc = SPH_OK;
    {
        std::vector<double> h(N);
        std::vector<uint32_t> tag(N);
        ParticleSet& S = c->set[0];
        auto upload = [&](double* dst, int which) -> cudaError_t {
            for (int a = 0; a < n_arrays; ++a) {
                const sph_array_desc& A = arrays[a];
                const double* src = nullptr;
                switch (which) {
                    case 0: src = A.x; break;
                    case 1: src = A.y; break;
                    case 2: src = A.z; break;
                    case 3: src = A.u; break;
                    case 4: src = A.v; break;
                    case 5: src = A.w; break;
                    case 6: src = A.rho; break;
                    default: src = A.m; break;
                }
                if ((which == 2 || which == 5) && domain->dim == 2) src = nullptr;
                for (int64_t i = 0; i < A.n; ++i) h[c->arr_off[a] + i] = src ? src[i] : 0.0;
            }
            return cudaMemcpyAsync(dst, h.data(), N * 8, cudaMemcpyHostToDevice, c->stream);
        };
        cudaError_t ue = cudaSuccess;
        double* dsts[8] = {S.x[0], S.x[1], S.x[2], S.u[0], S.u[1], S.u[2], S.rho, S.m};
        for (int k = 0; k < 8 && ue == cudaSuccess; ++k) {
            ue = upload(dsts[k], k);
            if (ue == cudaSuccess) ue = cudaStreamSynchronize(c->stream);
        }
        for (int a = 0; a < n_arrays; ++a) {
            for (int64_t i = 0; i < arrays[a].n; ++i)
                tag[c->arr_off[a] + i] = (uint32_t)(c->arr_off[a] + i) |
                                         (arrays[a].role == SPH_ROLE_WALL ? WALL_BIT : 0u);
            if (arrays[a].role == SPH_ROLE_WALL) c->nwall += (int)arrays[a].n;
        }
        if (ue == cudaSuccess)
            ue = cudaMemcpyAsync(S.tag, tag.data(), N * 4, cudaMemcpyHostToDevice, c->stream);
        // zero rates and the unused axes of both sets, the control block and the history
        for (int k = 0; k < 2 && ue == cudaSuccess; ++k) {
            ParticleSet& T = c->set[k];
            double* zs[8] = {T.arho, T.a[0], T.a[1], T.a[2], T.xs[0], T.xs[1], T.xs[2], T.p};
            for (double* z : zs)
                if (ue == cudaSuccess) ue = cudaMemsetAsync(z, 0, N * 8, c->stream);
            if (k == 1) {
                double* zz[8] = {T.x[0], T.x[1], T.x[2], T.u[0], T.u[1], T.u[2], T.rho, T.m};
                for (double* z : zz)
                    if (ue == cudaSuccess) ue = cudaMemsetAsync(z, 0, N * 8, c->stream);
            }
        }
        if (ue == cudaSuccess) ue = cudaMemsetAsync(c->ctl, 0, sizeof(Control), c->stream);
        if (ue == cudaSuccess) ue = cudaMemsetAsync(c->history, 0, (size_t)HIST_CAP * DIAG_N * 8, c->stream);
        if (ue == cudaSuccess && ninst == 0) {
            launch_wrap_all(c->set[0], c->N, c->G, c->stream, c->sms);
            ue = cudaGetLastError();
        }
        for (int k = 0; k < ninst && ue == cudaSuccess; ++k) {  // each instance in its box
            ParticleSet sub = c->set[0];
            const uint32_t f = c->id_bounds_h[k];
            for (int d = 0; d < 3; ++d) sub.x[d] += f;
            launch_wrap_all(sub, (int)(c->id_bounds_h[k + 1] - f), c->grids[k], c->stream, c->sms);
            ue = cudaGetLastError();
        }
        if (ue == cudaSuccess) {
            ue = cudaMemcpyAsync(c->d_id_bounds, c->id_bounds_h.data(), (nt + 1) * 4,
                                 cudaMemcpyHostToDevice, c->stream);
            if (ue == cudaSuccess)
                ue = cudaMemcpyAsync(c->d_cell_bounds, c->cell_bounds_h.data(), (nt + 1) * 4,
                                     cudaMemcpyHostToDevice, c->stream);
            if (ue == cudaSuccess) ue = cudaStreamSynchronize(c->stream);
        }
        if (ninst > 0 && ue == cudaSuccess) {
            if (ue == cudaSuccess) ue = cudaMemsetAsync(c->irec, 0, (size_t)ninst * DIAG_N * 8, c->stream);
            if (ue == cudaSuccess) ue = cudaMemsetAsync(c->it, 0, (size_t)ninst * 8, c->stream);
            if (ue == cudaSuccess) ue = cudaStreamSynchronize(c->stream);
        }
        if (ue == cudaSuccess) ue = cudaStreamSynchronize(c->stream);
        if (ue != cudaSuccess) {
            g_create_error = std::string("upload: ") + cudaGetErrorString(ue);
            rc = SPH_ERR_CUDA;
        }
    }
    if (rc != SPH_OK) {
        sph_destroy(c);
        return rc;
    }
    *out = c;
    return SPH_OK;
}

// ---------------------------------------------------------------- batches
sph_status grow_list(sph_ctx* c, int want) {
    void* p = nullptr;
    const size_t bytes = (size_t)want * c->N * 4;
    if (c->alloc) p = c->alloc(bytes, c->user);
    else if (cudaMalloc(&p, bytes) != cudaSuccess) p = nullptr;
    if (!p) {
        cudaGetLastError();
        return fail(c, SPH_ERR_OOM, "neighbour list of " + std::to_string(bytes) + " bytes");
    }
    CK(cudaStreamSynchronize(c->stream));
    free_dev(c, c->nl);
    c->nl = (uint32_t*)p;
    c->maxn = want;
    drop_graphs(c);
    return SPH_OK;
}

// Initial evaluation of every instance; the neighbour list grows until it holds the
// largest neighbourhood twice over (+32).
sph_status batch_initial_eval(sph_ctx* c) {
    if (!c->nl) {
        sph_status s = grow_list(c, c->dom.dim == 2 ? 64 : 256);
        if (s != SPH_OK) return s;
    }
    enqueue_build(c, 0, 0, 0);
    for (int attempt = 0; attempt < 8; ++attempt) {
        enqueue_eval(c, 0);
        unsigned status = 0;
        CK(cudaMemcpyAsync(&status, &c->ctl->status, sizeof status, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        if (!(status & ST_CAPACITY)) break;
        CK(cudaMemsetAsync(&c->ctl->status, 0, sizeof(unsigned), c->stream));
        c->work_dirty = true;
        sph_status s = grow_list(c, c->maxn * 2);
        if (s != SPH_OK) return s;
    }
    std::vector<uint32_t> counts(c->N);
    CK(cudaMemcpyAsync(counts.data(), c->cnt, (size_t)c->N * 4, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    uint32_t mx = 0;
    for (uint32_t v : counts) mx = v > mx ? v : mx;
    if ((uint32_t)c->maxn < 2 * mx + 32) {
        sph_status s = grow_list(c, (int)((2 * mx + 32 + 31) / 32 * 32));
        if (s != SPH_OK) return s;
    }
    c->have_rates = true;
    c->nbr_valid = true;
    return SPH_OK;
}

// The control block after a load: zeroed (status, counters, barrier words, stamps), then
// the saved time, step size and step count.
__global__ void k_load_control(Control* ctl, double t, double dt, unsigned long long step) {
    unsigned long long* w = reinterpret_cast<unsigned long long*>(ctl);
    for (size_t k = threadIdx.x; k < sizeof(Control) / 8; k += blockDim.x) w[k] = 0ull;
    __syncthreads();
    if (threadIdx.x == 0) {
        ctl->t = t;
        ctl->dt = dt;
        ctl->step = step;
    }
}

void launch_load_control(Control* ctl, double t, double dt, unsigned long long step, cudaStream_t st) {
    k_load_control<<<1, 64, 0, st>>>(ctl, t, dt, step);
}

// The step size of the next steps, set on the stream by value (a copy from host memory that
// is not pinned could make the host wait for the stream).
__global__ void k_set_dt(Control* ctl, double dt) { ctl->dt = dt; }

// State to / from a host buffer: the header's fixed part is written on the host, the time,
// step size and step count come from the control block by three small copies into the
// header, the fields by one copy each; `async` returns after enqueuing them.
sph_status save_state_impl(sph_ctx* c, void* buf, size_t* bytes, bool async) {
    if (!c || !bytes) return fail(c, SPH_ERR_INVALID, "NULL argument");
    const size_t N = (size_t)c->N;
    const size_t need = sizeof(StateHeader) + STATE_FIELDS * N * 8 + N * 4;
    if (!buf) {
        *bytes = need;
        return SPH_OK;
    }
    if (*bytes < need) {
        *bytes = need;
        return fail(c, SPH_ERR_CAPACITY, "state buffer too small");
    }
    StateHeader H{};
    H.magic = STATE_MAGIC;
    H.version = STATE_VERSION;
    H.n = c->N;
    H.dim = c->dom.dim;
    H.precision = c->dom.precision;
    H.have_rates = c->have_rates;
    H.scheme = c->rates_scheme;
    std::memcpy(buf, &H, sizeof H);
    StateHeader* hd = (StateHeader*)buf;
    CK(cudaMemcpyAsync(&hd->t, &c->ctl->t, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(&hd->dt, &c->ctl->dt, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(&hd->step, &c->ctl->step, sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                       c->stream));
    const ParticleSet& S = c->set[c->cur];
    double* fields[STATE_FIELDS];
    state_fields(S, fields);
    char* p = (char*)buf + sizeof(StateHeader);
    for (int k = 0; k < STATE_FIELDS; ++k)
        CK(cudaMemcpyAsync(p + (size_t)k * N * 8, fields[k], N * 8, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(p + STATE_FIELDS * N * 8, S.tag, N * 4, cudaMemcpyDeviceToHost, c->stream));
    if (!async) CK(cudaStreamSynchronize(c->stream));
    *bytes = need;
    return SPH_OK;
}

sph_status load_state_impl(sph_ctx* c, const void* buf, size_t bytes, bool async) {
    if (!c || !buf) return fail(c, SPH_ERR_INVALID, "NULL argument");
    const size_t N = (size_t)c->N;
    const size_t need = sizeof(StateHeader) + STATE_FIELDS * N * 8 + N * 4;
    StateHeader H;
    if (bytes < sizeof H) return fail(c, SPH_ERR_INVALID, "state buffer too small");
    std::memcpy(&H, buf, sizeof H);
    if (H.magic != STATE_MAGIC || H.version != STATE_VERSION || H.n != c->N || H.dim != c->dom.dim ||
        bytes < need)
        return fail(c, SPH_ERR_INVALID, "state buffer does not match this context");
    const ParticleSet& S = c->set[c->cur];
    double* fields[STATE_FIELDS];
    state_fields(S, fields);
    const char* p = (const char*)buf + sizeof(StateHeader);
    for (int k = 0; k < STATE_FIELDS; ++k)
        CK(cudaMemcpyAsync(fields[k], p + (size_t)k * N * 8, N * 8, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(S.tag, p + STATE_FIELDS * N * 8, N * 4, cudaMemcpyHostToDevice, c->stream));
    c->work_dirty = true;
    launch_load_control(c->ctl, H.t, H.dt, H.step, c->stream);  // the rest of the block zeroed
    CK(cudaGetLastError());
    if (!async) CK(cudaStreamSynchronize(c->stream));
    c->have_rates = H.have_rates != 0;
    c->rates_scheme = H.scheme;
    c->nbr_valid = false;
    c->hist_at_call = 0;
    c->steps_total = 0;
    return SPH_OK;
}

}  // namespace

extern "C" {

}  // extern "C"

namespace {

sph_status step_batch_impl(sph_ctx* c, const sph_scheme* schemes, const double* dt, int32_t nsteps,
                           bool sync) {
    if (!c) return fail(c, SPH_ERR_INVALID, "ctx is NULL");
    if (c->ninst == 0) return fail(c, SPH_ERR_STATE, "not a batch context");
    if (!schemes || !dt || nsteps < 0) return fail(c, SPH_ERR_INVALID, "bad arguments");
    bool changed = (int)c->batch_schemes.size() != c->ninst;
    for (int k = 0; k < c->ninst; ++k) {
        sph_status s = check_scheme(c, &schemes[k]);
        if (s != SPH_OK) return fail(c, s, "instance " + std::to_string(k) + ": " + c->err);
        if (schemes[k].density != schemes[0].density)
            return fail(c, SPH_ERR_INVALID, "instances must share the density formulation");
        if (schemes[k].integrator != schemes[0].integrator)
            return fail(c, SPH_ERR_INVALID, "instances must share the integrator");
        if (!std::isfinite(dt[k])) return fail(c, SPH_ERR_INVALID, "dt is not finite");
        if (!changed && (!same_scheme(schemes[k], c->batch_schemes[k]) || c->batch_dt[k] != dt[k]))
            changed = true;
    }
    if (changed) {
        c->batch_schemes.assign(schemes, schemes + c->ninst);
        c->batch_dt.assign(dt, dt + c->ninst);
        sph_status s = upload_table(c, schemes, dt);
        if (s != SPH_OK) return s;
        c->have_rates = false;
    }
    c->hist_at_call = c->steps_total;
    if (!c->have_rates) {
        // the initial evaluation's reduction sets every instance's next dt (the fixed dt of
        // the table, or the CFL-type criteria)
        sph_status s = batch_initial_eval(c);
        if (s != SPH_OK) return s;
    }
    if (nsteps > 0) {
        sph_status s = run_steps(c, nsteps);
        if (s != SPH_OK) return s;
        c->steps_total += (unsigned)nsteps;
        if (c->timing) c->timed_step_ran = true;
    }
    return sync ? sync_status(c) : SPH_OK;
}

}  // namespace

extern "C" {

sph_status sph_step_batch(sph_ctx* c, const sph_scheme* schemes, const double* dt, int32_t nsteps) {
    return step_batch_impl(c, schemes, dt, nsteps, true);
}

sph_status sph_step_batch_async(sph_ctx* c, const sph_scheme* schemes, const double* dt,
                                int32_t nsteps) {
    return step_batch_impl(c, schemes, dt, nsteps, false);
}

sph_status sph_batch_diagnostics(sph_ctx* c, double* out) {
    if (!c || !out) return fail(c, SPH_ERR_INVALID, "NULL argument");
    if (c->ninst == 0) return fail(c, SPH_ERR_STATE, "not a batch context");
    CK(cudaMemcpyAsync(out, c->irec, (size_t)c->ninst * DIAG_N * 8, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return SPH_OK;
}

}  // extern "C"

extern "C" {

sph_status sph_create(const sph_domain* domain, const sph_array_desc* arrays, int32_t n_arrays,
                      void* stream, sph_alloc_fn alloc, sph_free_fn free_fn, void* alloc_user,
                      sph_ctx** out) {
    return create_impl(domain, 0, arrays, nullptr, n_arrays, stream, alloc, free_fn, alloc_user, out);
}

sph_status sph_create_batch(const sph_domain* domains, const sph_array_desc* arrays,
                            const int32_t* arrays_per_instance, int32_t n_instances, void* stream,
                            sph_alloc_fn alloc, sph_free_fn free_fn, void* alloc_user,
                            sph_ctx** out) {
    if (n_instances < 1) return fail(nullptr, SPH_ERR_INVALID, "n_instances < 1");
    int32_t na = 0;
    if (arrays_per_instance)
        for (int k = 0; k < n_instances; ++k) na += arrays_per_instance[k];
    return create_impl(domains, n_instances, arrays, arrays_per_instance, na, stream, alloc, free_fn,
                       alloc_user, out);
}

void sph_destroy(sph_ctx* c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    drop_graphs(c);
    for (int k = 0; k < 7; ++k)
        if (c->ev[k]) cudaEventDestroy(c->ev[k]);
    free_dev(c, c->nl);
    free_dev(c, c->pec_save);
    free_dev(c, c->arena);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
}

const char* sph_last_error(const sph_ctx* c) {
    return c ? c->err.c_str() : g_create_error.c_str();
}

sph_status sph_count(const sph_ctx* ctx, int32_t array, int64_t* n) {
    sph_ctx* c = const_cast<sph_ctx*>(ctx);
    if (!c || !n) return fail(c, SPH_ERR_INVALID, "NULL argument");
    uint32_t first, count;
    sph_status s = array_range(c, array, &first, &count);
    if (s != SPH_OK) return s;
    *n = count;
    return SPH_OK;
}

sph_status sph_grid(const sph_ctx* ctx, int32_t n_cells[3], double cell_size[3], int64_t* ncells) {
    sph_ctx* c = const_cast<sph_ctx*>(ctx);
    if (!c || !n_cells || !cell_size || !ncells) return fail(c, SPH_ERR_INVALID, "NULL argument");
    for (int d = 0; d < 3; ++d) {
        n_cells[d] = c->G.nc[d];
        cell_size[d] = c->G.cs[d];
    }
    *ncells = c->G.ncells;
    return SPH_OK;
}

sph_status sph_build_neighbors(sph_ctx* c) {
    if (!c) return fail(c, SPH_ERR_INVALID, "ctx is NULL");
    if (c->ninst) return fail(c, SPH_ERR_STATE, "batch context: use the batch entry points");
    c->nbr_valid = false;
    sph_status s = ensure_neighbors(c);
    if (s != SPH_OK) return s;
    return sync_status(c);
}

sph_status sph_get_cells(sph_ctx* c, uint32_t* cell_of, uint32_t* offsets, int64_t* order) {
    if (!c || !cell_of || !offsets) return fail(c, SPH_ERR_INVALID, "NULL argument");
    if (c->ninst) return fail(c, SPH_ERR_STATE, "batch context: use the batch entry points");
    sph_status s = ensure_neighbors(c);
    if (s != SPH_OK) return s;
    uint32_t* d_cell = (uint32_t*)c->io;
    int64_t* d_order = (int64_t*)((char*)c->io + (((size_t)c->N * 4 + 255) & ~size_t(255)));
    launch_cell_of_by_id(c->skeys, c->set[c->cur].tag, c->N, d_cell, d_order, c->stream, c->sms);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(cell_of, d_cell, (size_t)c->N * 4, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(offsets, c->off, ((size_t)c->G.ncells + 1) * 4, cudaMemcpyDeviceToHost, c->stream));
    if (order)
        CK(cudaMemcpyAsync(order, d_order, (size_t)c->N * 8, cudaMemcpyDeviceToHost, c->stream));
    return sync_status(c);
}

sph_status sph_get_neighbors(sph_ctx* c, int64_t* offsets, int32_t* idx, int64_t* nnz) {
    if (!c || !offsets || !nnz) return fail(c, SPH_ERR_INVALID, "NULL argument");
    if (c->ninst) return fail(c, SPH_ERR_STATE, "batch context: use the batch entry points");
    sph_status s = ensure_neighbors(c);
    if (s != SPH_OK) return s;
    const PairConst<float> Kf = pair_const<float>(c, nullptr);
    const PairConst<double> Kd = pair_const<double>(c, nullptr);
    uint32_t* d_counts = (uint32_t*)c->io;
    launch_export_neighbors(c->dom.precision, c->dom.dim, c->P, c->skeys, c->off,
                            c->set[c->cur].tag, c->N, c->G, Kf, Kd, 0, d_counts, nullptr, nullptr,
                            c->stream, c->sms);
    CK(cudaGetLastError());
    std::vector<uint32_t> counts(c->N);
    CK(cudaMemcpyAsync(counts.data(), d_counts, (size_t)c->N * 4, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    offsets[0] = 0;
    for (int i = 0; i < c->N; ++i) offsets[i + 1] = offsets[i] + counts[i];
    const int64_t total = offsets[c->N];
    if (!idx) {
        *nnz = total;
        return SPH_OK;
    }
    if (*nnz < total) {
        *nnz = total;
        return fail(c, SPH_ERR_CAPACITY, "idx buffer too small");
    }
    *nnz = total;
    if (total == 0) return SPH_OK;
    int64_t* d_rows = (int64_t*)c->io;
    CK(cudaMemcpyAsync(d_rows, offsets, ((size_t)c->N + 1) * 8, cudaMemcpyHostToDevice, c->stream));
    void* d_idx = nullptr;
    if (c->alloc) d_idx = c->alloc((size_t)total * 4, c->user);
    else if (cudaMalloc(&d_idx, (size_t)total * 4) != cudaSuccess) d_idx = nullptr;
    if (!d_idx) {
        cudaGetLastError();
        return fail(c, SPH_ERR_OOM, "neighbour export buffer");
    }
    launch_export_neighbors(c->dom.precision, c->dom.dim, c->P, c->skeys, c->off,
                            c->set[c->cur].tag, c->N, c->G, Kf, Kd, 1, nullptr, d_rows,
                            (int32_t*)d_idx, c->stream, c->sms);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(idx, d_idx, (size_t)total * 4, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (c->free_fn) c->free_fn(d_idx, c->user);
    else cudaFree(d_idx);
    if (e != cudaSuccess) return cuda_fail(c, e, "neighbour export");
    return SPH_OK;
}

sph_status sph_eval_rhs(sph_ctx* c, const sph_scheme* scheme) {
    if (!c) return fail(c, SPH_ERR_INVALID, "ctx is NULL");
    if (c->ninst) return fail(c, SPH_ERR_STATE, "batch context: use the batch entry points");
    sph_status s = check_scheme(c, scheme);
    if (s != SPH_OK) return s;
    s = initial_eval(c, scheme, 0.0);
    if (s != SPH_OK) return s;
    return sync_status(c);
}

sph_status sph_step_async(sph_ctx* c, const sph_scheme* scheme, double dt, int32_t nsteps) {
    if (!c) return fail(c, SPH_ERR_INVALID, "ctx is NULL");
    if (c->ninst) return fail(c, SPH_ERR_STATE, "batch context: use the batch entry points");
    sph_status s = check_scheme(c, scheme);
    if (s != SPH_OK) return s;
    if (nsteps < 0) return fail(c, SPH_ERR_INVALID, "nsteps < 0");
    if (!std::isfinite(dt)) return fail(c, SPH_ERR_INVALID, "dt is not finite");
    if (dt <= 0.0) dt = 0.0;
    c->hist_at_call = c->steps_total;
    if (!c->have_rates || !same_scheme(*scheme, c->rates_scheme)) {
        s = initial_eval(c, scheme, dt);
        if (s != SPH_OK) return s;
    }
    if (!c->nl) {
        // a state loaded with its rates into a context that never evaluated: the neighbour
        // list is sized at the loaded positions (rates carried along, the order unchanged)
        s = ensure_neighbors(c);
        if (s != SPH_OK) return s;
        s = ensure_list_capacity(c);
        if (s != SPH_OK) return s;
    }
    s = upload_single(c, scheme, dt);
    if (s != SPH_OK) return s;
    if (dt > 0.0) {
        k_set_dt<<<1, 1, 0, c->stream>>>(c->ctl, dt);
        CK(cudaGetLastError());
    }
    if (nsteps == 0) return SPH_OK;
    s = run_steps(c, nsteps);
    if (s != SPH_OK) return s;
    c->steps_total += (unsigned)nsteps;
    c->nbr_valid = true;
    c->have_rates = true;
    if (c->timing) c->timed_step_ran = true;
    return SPH_OK;
}

sph_status sph_synchronize(sph_ctx* c) {
    if (!c) return fail(c, SPH_ERR_INVALID, "ctx is NULL");
    return sync_status(c);
}

sph_status sph_step(sph_ctx* c, const sph_scheme* scheme, double dt, int32_t nsteps) {
    sph_status s = sph_step_async(c, scheme, dt, nsteps);
    if (s != SPH_OK) return s;
    return sync_status(c);
}

sph_status sph_set_timing(sph_ctx* c, int32_t enable) {
    if (!c) return fail(c, SPH_ERR_INVALID, "ctx is NULL");
    if (enable && !c->ev[0])
        for (int k = 0; k < 7; ++k) CK(cudaEventCreate(&c->ev[k]));
    c->timing = enable != 0;
    return SPH_OK;
}

sph_status sph_phase_times(sph_ctx* c, float out[6]) {
    if (!c || !out) return fail(c, SPH_ERR_INVALID, "NULL argument");
    if (!c->timed_step_ran) return fail(c, SPH_ERR_STATE, "no timed step has run");
    if (c->last_fused) {  // phase-end stamps of the persistent kernel (block 0)
        Control h{};
        CK(cudaMemcpyAsync(&h, c->ctl, sizeof h, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        const unsigned long long* t = h.stamp;
        const double d[6] = {(double)(t[1] - t[0]), (double)(t[2] - t[1]), (double)(t[3] - t[2]),
                             0.0, (double)(t[4] - t[3]), (double)(t[6] - t[4])};
        for (int k = 0; k < 6; ++k) out[k] = (float)(d[k] * 1e-6);
        return SPH_OK;
    }
    if (!c->ev[0]) return fail(c, SPH_ERR_STATE, "no timed step has run");
    CK(cudaStreamSynchronize(c->stream));
    for (int k = 0; k < 6; ++k) CK(cudaEventElapsedTime(&out[k], c->ev[k], c->ev[k + 1]));
    return SPH_OK;
}

sph_status sph_kernels_per_step(const sph_ctx* ctx, const sph_scheme* scheme, int32_t* count) {
    sph_ctx* c = const_cast<sph_ctx*>(ctx);
    if (!c || !scheme || !count) return fail(c, SPH_ERR_INVALID, "NULL argument");
    // graph: keys + histograms, one launch per radix pass, reorder + cell table, density
    // pass, [solid-wall pressure], momentum pass (+ the two-stage per-instance reduction of
    // a batch); the midpoint integrator runs two of these and three stage kernels
    const bool wp = scheme->wall_bc == SPH_WALL_ADAMI && c->nwall > 0;
    const bool pec = scheme->integrator == SPH_INTEGRATOR_PEC;
    // (+ the chunk-partial finalize of a single problem's one-lane momentum pass with walls)
    const int build_eval = 1 + c->passes + 1 + 1 + (wp ? 1 : 0) + 1 + (c->ninst ? 2 : 0) +
                           (c->ninst == 0 && c->group_m == 1 && c->nwall > 0 ? 1 : 0);
    if (pec) *count = 2 * build_eval + 3;  // + predictor, corrector, record
    else *count = c->step_mode == SPH_STEP_PERSISTENT ? 1 : build_eval;
    return SPH_OK;
}

sph_status sph_set_groups(sph_ctx* c, int32_t momentum_lanes) {
    if (!c) return fail(c, SPH_ERR_INVALID, "ctx is NULL");
    if (momentum_lanes != 1 && momentum_lanes != 2 && momentum_lanes != 4 && momentum_lanes != 8)
        return fail(c, SPH_ERR_INVALID, "lanes per destination must be 1, 2, 4 or 8");
    set_groups(c, momentum_lanes, momentum_lanes);
    drop_graphs(c);
    return SPH_OK;
}

}  // extern "C"

namespace {

// Device copy of everything a few trial steps change (the current set, the control block,
// the batch's per-instance time, dt and records), to put the state back bitwise.
struct DevSnap {
    char* buf = nullptr;
    size_t bytes = 0;
};

size_t snap_bytes(const sph_ctx* c) {
    const size_t N = (size_t)c->N;
    return STATE_FIELDS * N * 8 + N * 4 + sizeof(Control) + (size_t)c->ninst * (2 + DIAG_N) * 8;
}

cudaError_t snap_copy(sph_ctx* c, const DevSnap& sn, bool restore) {
    const size_t N = (size_t)c->N;
    const ParticleSet& S = c->set[c->cur];
    double* f[STATE_FIELDS];
    state_fields(S, f);
    char* p = sn.buf;
    cudaError_t e = cudaSuccess;
    auto cp = [&](void* dev, size_t b) {
        if (e == cudaSuccess)
            e = restore ? cudaMemcpyAsync(dev, p, b, cudaMemcpyDeviceToDevice, c->stream)
                        : cudaMemcpyAsync(p, dev, b, cudaMemcpyDeviceToDevice, c->stream);
        p += b;
    };
    for (int k = 0; k < STATE_FIELDS; ++k) cp(f[k], N * 8);
    cp(S.tag, N * 4);
    cp(c->ctl, sizeof(Control));
    if (c->ninst) {
        cp(c->idt, (size_t)c->ninst * 8);
        cp(c->it, (size_t)c->ninst * 8);
        cp(c->irec, (size_t)c->ninst * DIAG_N * 8);
    }
    return e;
}

// Lanes per destination of each pair pass, timed pass by pass at the current state (the
// passes run without a kick: they act like an evaluation). The density pass of the chosen
// shape then leaves the lists the momentum pass is timed on.
sph_status tune_lanes(sph_ctx* c) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    const int reps = 5;
    auto time_it = [&](int pass, float* ms) -> cudaError_t {
        const StepLaunch L = step_launch(c, 0);
        for (int r = 0; r <= reps; ++r) {
            if (r == 1) cudaEventRecord(e0, c->stream);
            if (pass == 0) launch_density_pass(L, c->stream);
            else launch_momentum_pass(L, c->stream);
        }
        cudaEventRecord(e1, c->stream);
        cudaError_t e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
        return e;
    };
    int best[2] = {c->group_d, c->group_m};
    cudaError_t e = cudaSuccess;
    for (int pass = 0; pass < 2 && e == cudaSuccess; ++pass) {
        float best_ms = 1e30f;
        for (int T = 1; T <= 8 && e == cudaSuccess; T *= 2) {
            if (pass == 0) set_groups(c, T, c->group_m);
            else set_groups(c, best[0], T);
            float ms = 0.f;
            e = time_it(pass, &ms);
            if (e == cudaSuccess && ms < best_ms) {
                best_ms = ms;
                best[pass] = T;
            }
        }
        set_groups(c, best[0], pass == 0 ? c->group_m : best[1]);
        if (pass == 0 && e == cudaSuccess) {  // lists of the chosen density shape
            launch_density_pass(step_launch(c, 0), c->stream);
            e = cudaGetLastError();
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_fail(c, e, "autotune of the tile shapes");
    set_groups(c, best[0], best[1]);
    drop_graphs(c);
    return SPH_OK;
}

// Times a few steps in each mode from the same state and keeps the faster mode; the
// state, time and records are put back afterwards.
sph_status choose_mode(sph_ctx* c) {
    if (c->fused_bps[tindex(c->group_m)] < 1 || c->pec) {  // graph only
        c->step_mode = SPH_STEP_GRAPH;
        return SPH_OK;
    }
    int coop = 0;
    CK(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, c->device));
    if (!coop) {
        c->step_mode = SPH_STEP_GRAPH;
        return SPH_OK;
    }
    DevSnap sn;
    sn.bytes = snap_bytes(c);
    void* mem = nullptr;
    if (c->alloc) mem = c->alloc(sn.bytes, c->user);
    else if (cudaMalloc(&mem, sn.bytes) != cudaSuccess) mem = nullptr;
    if (!mem) {
        cudaGetLastError();
        return fail(c, SPH_ERR_OOM, "autotune snapshot of " + std::to_string(sn.bytes) + " bytes");
    }
    sn.buf = (char*)mem;
    const int cur0 = c->cur;
    uint32_t* skeys0 = c->skeys;
    const bool fused0 = c->last_fused;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    sph_status st = SPH_OK;
    float ms[2] = {0.f, 0.f};
    cudaError_t e = snap_copy(c, sn, false);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    for (int mode = 0; mode < 2 && e == cudaSuccess && st == SPH_OK; ++mode) {
        c->step_mode = mode;
        st = run_steps(c, 2);  // warm-up (and graph capture)
        if (st == SPH_OK) e = cudaEventRecord(e0, c->stream);
        if (st == SPH_OK && e == cudaSuccess) st = run_steps(c, 6);
        if (st == SPH_OK && e == cudaSuccess) e = cudaEventRecord(e1, c->stream);
        if (st == SPH_OK && e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (st == SPH_OK && e == cudaSuccess) e = cudaEventElapsedTime(&ms[mode], e0, e1);
        // back to the starting state
        c->cur = cur0;
        c->skeys = skeys0;
        if (e == cudaSuccess) e = snap_copy(c, sn, true);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    }
    c->last_fused = fused0;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaStreamSynchronize(c->stream);
    free_dev(c, mem);
    if (e != cudaSuccess) return cuda_fail(c, e, "autotune of the step mode");
    if (st != SPH_OK) return st;
    c->step_mode = ms[1] < ms[0] ? SPH_STEP_PERSISTENT : SPH_STEP_GRAPH;
    return SPH_OK;
}

}  // namespace

extern "C" {

sph_status sph_set_step_mode(sph_ctx* c, int32_t mode) {
    if (!c) return fail(c, SPH_ERR_INVALID, "ctx is NULL");
    if (mode != SPH_STEP_GRAPH && mode != SPH_STEP_PERSISTENT)
        return fail(c, SPH_ERR_INVALID, "unknown step mode");
    if (mode == SPH_STEP_PERSISTENT) {
        int coop = 0;
        CK(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, c->device));
        if (!coop) return fail(c, SPH_ERR_INVALID, "the device has no cooperative launch");
    }
    c->step_mode = mode;
    return SPH_OK;
}

sph_status sph_get_tuning(const sph_ctx* c, int32_t* momentum_lanes, int32_t* mode,
                          int32_t* density_lanes) {
    if (!c) return fail(nullptr, SPH_ERR_INVALID, "ctx is NULL");
    if (momentum_lanes) *momentum_lanes = c->group_m;
    if (mode) *mode = c->step_mode;
    if (density_lanes) *density_lanes = c->group_d;
    return SPH_OK;
}

sph_status sph_set_wait_limit(sph_ctx* c, uint64_t ns) {
    if (!c) return fail(c, SPH_ERR_INVALID, "ctx is NULL");
    c->wait_ns = ns;
    drop_graphs(c);  // the captured steps hold the limit
    return SPH_OK;
}

sph_status sph_autotune(sph_ctx* c, const sph_scheme* scheme, int32_t* chosen) {
    if (!c) return fail(c, SPH_ERR_INVALID, "ctx is NULL");
    if (c->ninst) {  // batch: the passes over all instances
        if ((int)c->batch_schemes.size() != c->ninst)
            return fail(c, SPH_ERR_STATE, "call sph_step_batch once before tuning a batch");
        sph_status s = batch_initial_eval(c);
        if (s != SPH_OK) return s;
        s = tune_lanes(c);
        if (s != SPH_OK) return s;
        s = sync_status(c);
        if (s != SPH_OK) return s;
        s = choose_mode(c);
        if (s != SPH_OK) return s;
        drop_graphs(c);
        if (chosen) *chosen = c->group_m;
        return sync_status(c);
    }
    sph_status s = check_scheme(c, scheme);
    if (s != SPH_OK) return s;
    s = initial_eval(c, scheme, 0.0);  // neighbours, list and a density pass at this state
    if (s != SPH_OK) return s;
    s = sync_status(c);
    if (s != SPH_OK) return s;
    s = tune_lanes(c);
    if (s != SPH_OK) return s;
    s = initial_eval(c, scheme, 0.0);  // rates and diagnostics of the chosen shape
    if (s != SPH_OK) return s;
    s = sync_status(c);
    if (s != SPH_OK) return s;
    s = choose_mode(c);
    if (s != SPH_OK) return s;
    drop_graphs(c);
    remember_tuning(c);
    if (chosen) *chosen = c->group_m;
    return sync_status(c);
}

// ------------------------------------------------------------------- adjoint
namespace {

// Snapshot of the FP64 state of the current set (x, u, rho, m, arho, a, xsph, tag).
struct Snapshot {
    double* f[15];
    uint32_t* tag;
};

void snap_take(sph_ctx* c, char*& p, Snapshot& sn) {
    for (int k = 0; k < 15; ++k) sn.f[k] = (double*)arena_take(p, (size_t)c->N * 8);
    sn.tag = (uint32_t*)arena_take(p, (size_t)c->N * 4);
}

void set_fields(const ParticleSet& S, double* const* f_in, double** f_out) {
    double* fs[15] = {S.x[0], S.x[1], S.x[2], S.u[0], S.u[1], S.u[2], S.rho, S.m,
                      S.arho, S.a[0], S.a[1], S.a[2], S.xs[0], S.xs[1], S.xs[2]};
    (void)f_in;
    for (int k = 0; k < 15; ++k) f_out[k] = fs[k];
}

cudaError_t snap_save(sph_ctx* c, const Snapshot& sn) {
    double* fs[15];
    set_fields(c->set[c->cur], nullptr, fs);
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 15 && e == cudaSuccess; ++k)
        e = cudaMemcpyAsync(sn.f[k], fs[k], (size_t)c->N * 8, cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(sn.tag, c->set[c->cur].tag, (size_t)c->N * 4, cudaMemcpyDeviceToDevice,
                            c->stream);
    return e;
}

cudaError_t snap_load(sph_ctx* c, const Snapshot& sn) {
    double* fs[15];
    set_fields(c->set[c->cur], nullptr, fs);
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 15 && e == cudaSuccess; ++k)
        e = cudaMemcpyAsync(fs[k], sn.f[k], (size_t)c->N * 8, cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->set[c->cur].tag, sn.tag, (size_t)c->N * 4, cudaMemcpyDeviceToDevice,
                            c->stream);
    return e;
}

// Taped evaluation: the pair-loop shadow after its density pass, the permutation to the
// previous order and the tags, all in the evaluation's cell order.
struct TapeEntry {
    void* P;
    void* Q;
    void* R;
    uint32_t* perm;
    uint32_t* tag;
    uint32_t* nl;   // neighbour list of the evaluation (maxn x N words, interleaved)
    uint32_t* cnt;
};

void tape_take(sph_ctx* c, char*& p, TapeEntry& t) {
    const size_t real = c->dom.precision ? 4 : 8;
    t.P = arena_take(p, (size_t)c->N * 4 * real);
    t.Q = arena_take(p, (size_t)c->N * 4 * real);
    t.R = arena_take(p, (size_t)c->N * real);
    t.perm = (uint32_t*)arena_take(p, (size_t)c->N * 4);
    t.tag = (uint32_t*)arena_take(p, (size_t)c->N * 4);
    t.nl = (uint32_t*)arena_take(p, (size_t)c->maxn * c->N * 4);
    t.cnt = (uint32_t*)arena_take(p, (size_t)c->N * 4);
}

cudaError_t tape_record(sph_ctx* c, const TapeEntry& t) {
    const size_t real = c->dom.precision ? 4 : 8;
    const size_t N = (size_t)c->N;
    cudaError_t e = cudaMemcpyAsync(t.P, c->P, N * 4 * real, cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(t.Q, c->Q, N * 4 * real, cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(t.R, c->R, N * real, cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(t.perm, c->vals[c->passes & 1], N * 4, cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(t.tag, c->set[c->cur].tag, N * 4, cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess) {
        launch_tape_list(c->nl, c->cnt, c->N, t.nl, t.cnt, c->sms, c->stream);
        e = cudaGetLastError();
    }
    return e;
}

AdjSet adj_take(sph_ctx* c, char*& p) {
    AdjSet L{};
    for (int d = 0; d < 3; ++d) L.x[d] = (double*)arena_take(p, (size_t)c->N * 8);
    for (int d = 0; d < 3; ++d) L.u[d] = (double*)arena_take(p, (size_t)c->N * 8);
    L.rho = (double*)arena_take(p, (size_t)c->N * 8);
    for (int d = 0; d < 3; ++d) L.a[d] = (double*)arena_take(p, (size_t)c->N * 8);
    for (int d = 0; d < 3; ++d) L.xs[d] = (double*)arena_take(p, (size_t)c->N * 8);
    return L;
}

}  // namespace

sph_status sph_backward(sph_ctx* c, const sph_scheme* scheme, double dt, int32_t K,
                        int32_t ckpt_every, double* dKE_du0, double* dKE_dnu, double* dKE_dalpha) {
    if (!c) return fail(c, SPH_ERR_INVALID, "ctx is NULL");
    if (c->ninst) return fail(c, SPH_ERR_STATE, "batch context: use the batch entry points");
    sph_status s = check_scheme(c, scheme);
    if (s != SPH_OK) return s;
    if (scheme->density != SPH_DENSITY_CONTINUITY)
        return fail(c, SPH_ERR_INVALID, "the adjoint covers the continuity formulation only");
    if (scheme->wall_bc != SPH_WALL_DENSITY)
        return fail(c, SPH_ERR_INVALID, "the adjoint does not cover the solid-wall pressure");
    if (scheme->integrator != SPH_INTEGRATOR_KDK)
        return fail(c, SPH_ERR_INVALID, "the adjoint covers the kick-drift-kick integrator only");
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(c, SPH_ERR_INVALID, "the adjoint needs a fixed dt > 0");
    if (K < 0) return fail(c, SPH_ERR_INVALID, "K < 0");
    int C = ckpt_every;
    if (C <= 0) C = (int)std::ceil(std::sqrt((double)(K > 0 ? K : 1)));
    if (C > K && K > 0) C = K;
    if (C < 1) C = 1;
    const int nseg = K > 0 ? (K + C - 1) / C : 0;
    // initial evaluation first: it sizes the neighbour list that the tape copies
    s = initial_eval(c, scheme, dt);
    if (s != SPH_OK) return s;
    const size_t N = (size_t)c->N;
    const size_t real = c->dom.precision ? 4 : 8;
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    const int pblocks = adjoint_partial_blocks(c->N, c->sms);
    size_t bytes = 0;
    bytes += (size_t)(nseg + 1) * (15 * al(N * 8) + al(N * 4));                 // checkpoints + final
    bytes += (size_t)(C + 1) * (2 * al(N * 4 * real) + al(N * real) + 3 * al(N * 4) +
                                al((size_t)c->maxn * N * 4));                      // tape
    bytes += 2 * 13 * al(N * 8) + 5 * al(N * 8) + 2 * al(N * 4 * real);         // adjoint state
    bytes += al(N * 8 * 3) + al((size_t)pblocks * 16) + al(sizeof(AdjCtl));
    void* arena = nullptr;
    if (c->alloc) arena = c->alloc(bytes, c->user);
    else if (cudaMalloc(&arena, bytes) != cudaSuccess) arena = nullptr;
    if (!arena) {
        cudaGetLastError();
        return fail(c, SPH_ERR_OOM, "adjoint workspace of " + std::to_string(bytes) + " bytes");
    }
    struct Guard {
        sph_ctx* c;
        void* p;
        ~Guard() {
            cudaStreamSynchronize(c->stream);
            free_dev(c, p);
        }
    } guard{c, arena};
    char* p = (char*)arena;
    std::vector<Snapshot> ck(nseg + 1);
    for (auto& sn : ck) snap_take(c, p, sn);  // ck[nseg] holds the final state
    std::vector<TapeEntry> tape(C + 1);       // tape[C] holds the initial evaluation
    for (auto& t : tape) tape_take(c, p, t);
    AdjSet L[2] = {adj_take(c, p), adj_take(c, p)};
    double* luh[3];
    for (int d = 0; d < 3; ++d) luh[d] = (double*)arena_take(p, N * 8);
    double* rhom = (double*)arena_take(p, N * 8);
    double* lrho_tot = (double*)arena_take(p, N * 8);
    void* CA = arena_take(p, N * 4 * real);
    void* CS = arena_take(p, N * 4 * real);
    double* d_out = (double*)arena_take(p, N * 8 * 3);
    double* part = (double*)arena_take(p, (size_t)pblocks * 16);
    AdjCtl* actl = (AdjCtl*)arena_take(p, sizeof(AdjCtl));
    CK(cudaMemsetAsync(actl, 0, sizeof(AdjCtl), c->stream));
    CK(cudaMemsetAsync(d_out, 0, N * 8 * 3, c->stream));

    // ---- forward: initial evaluation (taped) and checkpoints every C steps
    CK(cudaMemcpyAsync(&c->ctl->dt, &dt, sizeof dt, cudaMemcpyHostToDevice, c->stream));
    CK(tape_record(c, tape[C]));
    if (!c->graph[0] || c->graph_timed != c->timing) {
        s = capture_step_graphs(c);
        if (s != SPH_OK) return s;
    }
    // segments end-aligned: segment 0 holds the remainder (1..C steps), the others C steps;
    // the last segment is taped during this sweep (it is reversed first, so it is never
    // recomputed), the others are recomputed from their checkpoints
    auto seg_begin = [&](int sg) { return sg == 0 ? 0 : K - (nseg - sg) * C; };
    const int taped0 = nseg > 0 ? seg_begin(nseg - 1) : K;
    CK(clear_work_if_dirty(c));
    for (int sg = 0, step = 0; step < K; ++step) {
        if (sg < nseg - 1 && step == seg_begin(sg)) CK(snap_save(c, ck[sg++]));
        CK(cudaGraphLaunch(c->graph[c->cur], c->stream));
        c->cur ^= 1;
        if (step >= taped0) CK(tape_record(c, tape[step - taped0]));
    }
    CK(snap_save(c, ck[nseg]));
    Control ctl_final{};
    CK(cudaMemcpyAsync(&ctl_final, c->ctl, sizeof ctl_final, cudaMemcpyDeviceToHost, c->stream));
    s = sync_status(c);
    if (s != SPH_OK) return s;

    // ---- reverse
    const StepConst Cst = step_const(c, scheme, dt);
    const PairConst<float> Kf = pair_const<float>(c, scheme);
    const PairConst<double> Kd = pair_const<double>(c, scheme);
    AdjLaunch A{};
    A.precision = c->dom.precision;
    A.dim = c->dom.dim;
    A.kernel = c->dom.kernel;
    A.n = c->N;
    A.sms = c->sms;
    A.dt = dt;
    A.G = c->G;
    A.C = Cst;
    for (int d = 0; d < 3; ++d) A.luh[d] = luh[d];
    A.rhom = rhom;
    A.lrho_tot = lrho_tot;
    A.CA = CA;
    A.CS = CS;
    A.part = part;
    A.actl = actl;
    int lc = 0;
    launch_adjoint_terminal(L[lc], c->set[c->cur], c->N, c->dom.dim, c->sms, c->stream);
    for (int seg = nseg - 1; seg >= 0; --seg) {
        const int s0 = seg_begin(seg), s1 = seg + 1 < nseg ? seg_begin(seg + 1) : K;
        if (seg < nseg - 1) {  // recompute from the checkpoint, taping each step
            CK(snap_load(c, ck[seg]));
            CK(cudaMemsetAsync(&c->ctl->status, 0, sizeof(unsigned), c->stream));
            c->work_dirty = true;
            CK(clear_work_if_dirty(c));
            CK(cudaMemcpyAsync(&c->ctl->dt, &dt, sizeof dt, cudaMemcpyHostToDevice, c->stream));
            for (int step = s0; step < s1; ++step) {
                CK(cudaGraphLaunch(c->graph[c->cur], c->stream));
                c->cur ^= 1;
                CK(tape_record(c, tape[step - s0]));
            }
        }
        for (int step = s1 - 1; step >= s0; --step) {
            const TapeEntry& t = tape[step - s0];
            A.P = t.P;
            A.Q = t.Q;
            A.R = t.R;
            A.perm = t.perm;
            A.tag = t.tag;
            A.nl = t.nl;
            A.cnt = t.cnt;
            A.kick = 1;
            A.L = L[lc];
            launch_adjoint_eval(A, Kf, Kd, c->stream);
            launch_adjoint_scatter(A, L[lc ^ 1], c->stream);
            lc ^= 1;
        }
        CK(cudaGetLastError());
    }
    // initial evaluation: (a0, xsph0) = M(x0, u0, rho0), no density update, no kick
    A.P = tape[C].P;
    A.Q = tape[C].Q;
    A.R = tape[C].R;
    A.perm = tape[C].perm;
    A.tag = tape[C].tag;
    A.nl = tape[C].nl;
    A.cnt = tape[C].cnt;
    A.kick = 0;
    A.L = L[lc];
    launch_adjoint_eval(A, Kf, Kd, c->stream);
    launch_adjoint_to_original(A, d_out, c->stream);
    CK(cudaGetLastError());
    AdjCtl actl_h{};
    CK(cudaMemcpyAsync(&actl_h, actl, sizeof actl_h, cudaMemcpyDeviceToHost, c->stream));
    if (dKE_du0)
        CK(cudaMemcpyAsync(dKE_du0, d_out, N * 8 * c->dom.dim, cudaMemcpyDeviceToHost, c->stream));
    // leave the context in the final state of the K steps
    CK(snap_load(c, ck[nseg]));
    CK(cudaMemcpyAsync(c->ctl, &ctl_final, sizeof ctl_final, cudaMemcpyHostToDevice, c->stream));
    s = sync_status(c);
    if (s != SPH_OK) return s;
    c->nbr_valid = false;
    c->have_rates = true;
    c->rates_scheme = *scheme;
    c->hist_at_call = c->steps_total;
    c->steps_total += (unsigned)K;
    if (dKE_dnu) *dKE_dnu = actl_h.g_nu;
    if (dKE_dalpha) *dKE_dalpha = actl_h.g_alpha;
    return SPH_OK;
}

sph_status sph_get(sph_ctx* c, int32_t array, const char* prop, double* out) {
    if (!c || !out) return fail(c, SPH_ERR_INVALID, "NULL argument");
    double* field = nullptr;
    sph_status s = prop_field(c, prop, false, &field);
    if (s != SPH_OK) return s;
    uint32_t first, count;
    s = array_range(c, array, &first, &count);
    if (s != SPH_OK) return s;
    if (count == 0) return SPH_OK;
    double* d_out = (double*)c->io;
    launch_gather_by_id(field, c->set[c->cur].tag, c->N, first, count, d_out, c->stream, c->sms);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(out, d_out, (size_t)count * 8, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return SPH_OK;
}

sph_status sph_set(sph_ctx* c, int32_t array, const char* prop, const double* in) {
    if (!c || !in) return fail(c, SPH_ERR_INVALID, "NULL argument");
    double* field = nullptr;
    sph_status s = prop_field(c, prop, true, &field);
    if (s != SPH_OK) return s;
    uint32_t first, count;
    s = array_range(c, array, &first, &count);
    if (s != SPH_OK) return s;
    if (count == 0) return SPH_OK;
    double* d_in = (double*)c->io;
    CK(cudaMemcpyAsync(d_in, in, (size_t)count * 8, cudaMemcpyHostToDevice, c->stream));
    launch_scatter_by_id(field, c->set[c->cur].tag, c->N, first, count, d_in, c->stream, c->sms);
    if (prop[0] == 'x' || prop[0] == 'y' || prop[0] == 'z')
        launch_wrap_all(c->set[c->cur], c->N, c->G, c->stream, c->sms);
    CK(cudaGetLastError());
    CK(cudaMemsetAsync(&c->ctl->status, 0, sizeof(unsigned), c->stream));
        c->work_dirty = true;
    CK(cudaStreamSynchronize(c->stream));
    c->have_rates = false;
    c->nbr_valid = false;
    return SPH_OK;
}

sph_status sph_diagnostics(sph_ctx* c, double* out) {
    if (!c || !out) return fail(c, SPH_ERR_INVALID, "NULL argument");
    CK(cudaMemcpyAsync(out, c->ctl->rec, DIAG_N * 8, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return SPH_OK;
}

sph_status sph_history(sph_ctx* c, double* out, int32_t max_records, int32_t* count) {
    if (!c || !out || !count || max_records < 0) return fail(c, SPH_ERR_INVALID, "bad argument");
    unsigned end = 0;
    CK(cudaMemcpyAsync(&end, &c->ctl->hist_count, sizeof end, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    unsigned begin = c->hist_at_call;
    unsigned avail = end >= begin ? end - begin : 0u;
    if (avail > (unsigned)HIST_CAP) {
        begin = end - HIST_CAP;
        avail = HIST_CAP;
    }
    unsigned n = avail < (unsigned)max_records ? avail : (unsigned)max_records;
    unsigned done = 0;
    while (done < n) {  // at most two contiguous pieces of the ring
        unsigned slot = (begin + done) % HIST_CAP;
        unsigned piece = n - done;
        if (piece > HIST_CAP - slot) piece = HIST_CAP - slot;
        CK(cudaMemcpyAsync(out + (size_t)done * DIAG_N, c->history + (size_t)slot * DIAG_N,
                           (size_t)piece * DIAG_N * 8, cudaMemcpyDeviceToHost, c->stream));
        done += piece;
    }
    CK(cudaStreamSynchronize(c->stream));
    *count = (int32_t)n;
    return SPH_OK;
}

sph_status sph_save_state(sph_ctx* c, void* buf, size_t* bytes) {
    return save_state_impl(c, buf, bytes, false);
}

sph_status sph_save_state_async(sph_ctx* c, void* buf, size_t* bytes) {
    return save_state_impl(c, buf, bytes, true);
}

sph_status sph_load_state(sph_ctx* c, const void* buf, size_t bytes) {
    return load_state_impl(c, buf, bytes, false);
}

sph_status sph_load_state_async(sph_ctx* c, const void* buf, size_t bytes) {
    return load_state_impl(c, buf, bytes, true);
}

}  // extern "C"
