/*
 * sph.h - C ABI of a GB300-native implementation of the data-parallel hot path of
 * weakly-compressible SPH (WCSPH) as described in the PySPH paper: uniform-grid
 * neighbour search (cell keys, radix sort, reorder, cell table; Sec. 2.2), the fused
 * pair loops (summation density Eq. 2 or continuity Eq. continuity:sph, Tait EOS
 * Eq. eos, momentum Eqs. mom:sph, mom:sph:press, mom:sph:visc with Monaghan
 * artificial viscosity and XSPH; quintic spline and Wendland C2 kernels) and the
 * predictor-corrector integrator of Sec. 2.1 with periodic wrap and static wall
 * particles.
 *
 * Conventions shared by every entry point:
 *  - Every call returns an sph_status; nothing aborts, traps or exits. On failure the
 *    message is available from sph_last_error().
 *  - Host pointers ("host") are read or written only during the call. Device memory
 *    belongs to the context (allocated through the caller's allocator, or cudaMalloc
 *    when none is given) and is released by sph_destroy().
 *  - Particle ids are global: the arrays given to sph_create are concatenated in order,
 *    so array a, local index i has global id offset(a) + i. Every per-particle output
 *    is in that original order, whatever order the device keeps internally.
 *  - All device work is issued on the stream given at creation. Calls that return data
 *    to the host synchronise that stream. A context is used from one thread at a time.
 */
#ifndef SPH_H
#define SPH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sph_ctx sph_ctx;

typedef enum {
    SPH_OK = 0,
    SPH_ERR_INVALID = 1,    /* an argument is out of range or inconsistent */
    SPH_ERR_CUDA = 2,       /* a CUDA runtime call or a kernel launch failed */
    SPH_ERR_OOM = 3,        /* the allocator returned NULL */
    SPH_ERR_NONFINITE = 4,  /* a step produced NaN/Inf; later steps of the call were skipped */
    SPH_ERR_DOMAIN = 5,     /* reserved: particle outside the cell box (such particles are
                               clamped into the edge cells and counted, not rejected) */
    SPH_ERR_CAPACITY = 6,   /* a caller buffer or a fixed capacity is too small */
    SPH_ERR_TIMEOUT = 7,    /* a bounded device-side wait gave up */
    SPH_ERR_STATE = 8       /* the call is not valid in the context's current state */
} sph_status;

typedef enum { SPH_KERNEL_QUINTIC = 0, SPH_KERNEL_WENDLAND_C2 = 1, SPH_KERNEL_CUBIC_SPLINE = 2 } sph_kernel;
typedef enum { SPH_PREC_FP64 = 0, SPH_PREC_FP32 = 1 } sph_precision;
typedef enum { SPH_ROLE_FLUID = 0, SPH_ROLE_WALL = 1 } sph_role;
typedef enum { SPH_DENSITY_CONTINUITY = 0, SPH_DENSITY_SUMMATION = 1, SPH_DENSITY_EDAC = 2 } sph_density;
typedef enum { SPH_WALL_DENSITY = 0, SPH_WALL_ADAMI = 1 } sph_wall_bc;
typedef enum { SPH_INTEGRATOR_KDK = 0, SPH_INTEGRATOR_PEC = 1 } sph_integrator;

/* Geometry of a problem (Sec. 2.2, Sec. 3 create_domain).
 *  dim        2 or 3.
 *  kernel     sph_kernel: quintic spline (support 3h), Wendland C2 (support 2h) or the
 *             cubic (M4) B-spline (support 2h).
 *  precision  sph_precision of the pair loops. FP32: positions are rounded once to
 *             float and the neighbour test and pair sums run in float with compensated
 *             (Neumaier) per-particle sums; the integrator, the state and the
 *             reductions stay FP64. FP64: everything in double.
 *  periodic   per axis; a periodic axis wraps positions into [lo, hi) and uses the
 *             minimum image in the neighbour test. It needs at least 2 R + 1 cells.
 *  h          smoothing length (constant for all particles).
 *  lo, hi     cell box. On a periodic axis it is the period. Cells per axis:
 *             n = floor((hi - lo) / (k h / R * 1.00001)), size (hi - lo) / n, with k the
 *             support factor and R = 1 in 2D, 2 in 3D (a (2R + 1)^dim cell stencil); a particle outside the box on a non-periodic axis is
 *             clamped into the edge cell (the result stays exact, only slower). */
typedef struct {
    int32_t dim;
    int32_t kernel;
    int32_t precision;
    int32_t periodic[3];
    double h;
    double lo[3];
    double hi[3];
} sph_domain;

/* One named particle array (the ParticleArray of Sec. 3.2.1). Host pointers, copied at
 * creation, n entries each. z and w may be NULL in 2D; u, v, w may be NULL (zero).
 * x, y, rho, m are required. Wall particles never move: their x and u stay as given. */
typedef struct {
    const char* name;
    int32_t role;
    int64_t n;
    const double* x;
    const double* y;
    const double* z;
    const double* u;
    const double* v;
    const double* w;
    const double* rho;
    const double* m;
} sph_array_desc;

/* Equations of one right-hand-side evaluation (Sec. 3.2 groups: [summation density],
 * EOS, then continuity + momentum; walls take continuity from fluid sources only).
 *  density    sph_density. SPH_DENSITY_EDAC: the EDAC scheme of the scheme list of
 *             Sec. 2.3, with which Sec. 4.1 solves the Taylor-Green vortex: the pressure
 *             "p" is a particle variable, dp/dt = -rho0 c0^2 div u + nu_e lap p with
 *             nu_e = h c0 / 16 (the EDAC diffusivity alpha h c0 / 8 at alpha = 0.5), as
 *             dp_i/dt = c0^2 sum_j m_j u_ij . grad_i W_ij + (2 nu_e / rho0) sum_j m_j
 *             (p_i - p_j) (r_ij . grad_i W_ij) / (r_ij^2 + 0.01 h^2); the density stays
 *             rho0 (volumes m / rho0) and gamma is unused; the pressure is advanced like
 *             the continuity density in the step and read by the momentum equation.
 *             Fluid-only problems with the kick-drift-kick integrator (wall particles,
 *             SPH_INTEGRATOR_PEC and sph_backward are refused). The rate is read as
 *             "arho", the pressure as "p".
 *  rho0, c0, gamma   Tait EOS, Eq. eos: p = c0^2 rho0 / gamma ((rho/rho0)^gamma - 1).
 *  nu, eta    laminar viscosity, Eq. mom:sph:visc (term off when nu == 0).
 *  alpha      Monaghan artificial viscosity: Pi_ij = -alpha c0 mu_ij / rhobar_ij when
 *             v_ij . r_ij < 0, mu_ij = h v_ij . r_ij / (r^2 + 0.01 h^2) (off when 0).
 *  xsph_eps   XSPH: dx_i = eps sum_fluid j m_j / rhobar_ij (u_j - u_i) W_ij, added to the
 *             drift velocity (off when 0).
 *  g          body acceleration of fluid particles, Eq. mom:sph.
 *  wall_bc    sph_wall_bc. SPH_WALL_DENSITY: wall pressure from the wall density of the
 *             formulation (continuity from fluid sources, or summation). SPH_WALL_ADAMI:
 *             the solid-wall condition of Adami, Hu and Adams (2012), one of the wall
 *             boundary conditions listed among the schemes of Sec. 2.3: after the density
 *             pass each wall particle w takes p_w = (sum_f p_f W_wf + g . sum_f rho_f
 *             (x_w - x_f) W_wf) / sum_f W_wf over its fluid neighbours f (static walls)
 *             and rho_w = rho0 (1 + p_w / B)^(1/gamma), B = c0^2 rho0 / gamma; a wall
 *             with no fluid neighbour takes p_w = 0, rho_w = rho0. One more launch per
 *             evaluation (graph step form only; sph_backward rejects it).
 *  integrator sph_integrator. SPH_INTEGRATOR_KDK: the predictor-corrector of Sec. 2.1 as
 *             kick-drift-kick (u^{n+1/2} = u^n + dt/2 a^n, x^{n+1} = x^n + dt (u^{n+1/2}
 *             + xsph^n), rho^{n+1} = rho^n + dt arho(x^{n+1}, u^{n+1/2}), u^{n+1} =
 *             u^{n+1/2} + dt/2 a^{n+1}), one evaluation per step; second order for
 *             forces of the positions alone, first order where the rates depend on
 *             the velocity (viscosity, artificial viscosity, XSPH, the continuity
 *             rate), which it evaluates with u^{n+1/2}. SPH_INTEGRATOR_PEC: the
 *             two-evaluation midpoint predict-evaluate-correct form (Monaghan 2005),
 *             second order: a half step with the rates at t^n (u* = u^n + dt/2 a^n,
 *             x* = x^n + dt/2 (u^n + xsph^n), rho* = rho^n + dt/2 arho^n), an evaluation
 *             at the midpoint, the full step from t^n with the midpoint rates (u^{n+1} =
 *             u^n + dt a*, x^{n+1} = x^n + dt (u^n + dt/2 a* + xsph*), rho^{n+1} = rho^n +
 *             dt arho*), and an evaluation at t^{n+1}: two neighbour builds and two
 *             evaluations per step. Graph step form only; the instances of a batch
 *             share it; sph_backward rejects it.
 *  reserved   must be 0. */
typedef struct {
    int32_t density;
    int32_t wall_bc;
    int32_t integrator;
    int32_t reserved;
    double rho0;
    double c0;
    double gamma;
    double nu;
    double eta;
    double alpha;
    double xsph_eps;
    double g[3];
} sph_scheme;

/* Device allocator callbacks: return a device pointer of at least `bytes` bytes aligned
 * to 256 bytes (NULL on failure) / release it. Both may be NULL to use cudaMalloc. */
typedef void* (*sph_alloc_fn)(size_t bytes, void* user);
typedef void (*sph_free_fn)(void* ptr, void* user);

/* Diagnostics record layout (sph_diagnostics, sph_history). FP64 reductions over
 * fluid particles after the last right-hand-side evaluation (Sec. 2.1 criteria). */
enum {
    SPH_DIAG_T = 0,          /* simulated time */
    SPH_DIAG_DT = 1,         /* step used to reach it (0 for the initial evaluation) */
    SPH_DIAG_KE = 2,         /* 1/2 sum m |u|^2 */
    SPH_DIAG_UMAX = 3,       /* max |u| */
    SPH_DIAG_PX = 4,         /* sum m u (x, y, z) */
    SPH_DIAG_PY = 5,
    SPH_DIAG_PZ = 6,
    SPH_DIAG_AMAX = 7,       /* max |a| */
    SPH_DIAG_PAIRS = 8,      /* ordered interacting pairs i != j of the evaluation */
    SPH_DIAG_CANDIDATES = 9, /* ordered pairs examined in the 3^d cell stencil, j != i */
    SPH_DIAG_STEP = 10,      /* steps taken since creation */
    SPH_DIAG_OUTSIDE = 11,   /* particles clamped into an edge cell at the last build */
    SPH_DIAG_WALL_PAIRS = 12,/* of SPH_DIAG_PAIRS, those with a wall destination */
    SPH_DIAG_COUNT = 13
};

/* Create a context: copy the arrays to the device (global ids in array order), wrap
 * periodic coordinates into the box. `stream` is a cudaStream_t (NULL: the context creates
 * and owns a non-blocking stream, needed because steps run as captured CUDA graphs). Returns SPH_ERR_INVALID for a bad domain (dim, kernel, h <= 0, empty box,
 * a periodic axis with fewer than 3 cells, 2^30 particles or more). */
sph_status sph_create(const sph_domain* domain, const sph_array_desc* arrays, int32_t n_arrays,
                      void* stream, sph_alloc_fn alloc, sph_free_fn free_fn, void* alloc_user,
                      sph_ctx** out);

/* Release every device buffer and the context. NULL is ignored. */
void sph_destroy(sph_ctx* ctx);

/* Message of the last failed call on ctx (ctx NULL: of the last failed sph_create on this
 * thread). Valid until the next call on the same context. */
const char* sph_last_error(const sph_ctx* ctx);

/* Particle count of array `array` (-1: all particles). */
sph_status sph_count(const sph_ctx* ctx, int32_t array, int64_t* n);

/* Cell grid: cells per axis, cell sizes, total cells (Sec. 2.2). */
sph_status sph_grid(const sph_ctx* ctx, int32_t n_cells[3], double cell_size[3], int64_t* ncells);

/* Neighbour build at the current positions (Sec. 2.2, Z-order/cell sort): cell key per
 * particle, stable radix sort, reorder of the state into cell order and the cell table. */
sph_status sph_build_neighbors(sph_ctx* ctx);

/* Cell table of the last build, host buffers. cell_of (n_total, original order): linear
 * cell id cx + nx (cy + ny cz). offsets (ncells + 1): offsets[c] = particles in cells < c,
 * so cell c holds sorted positions [offsets[c], offsets[c+1]). order (n_total, may be
 * NULL): global id at each sorted position. Builds first if positions changed. */
sph_status sph_get_cells(sph_ctx* ctx, uint32_t* cell_of, uint32_t* offsets, int64_t* order);

/* Neighbour lists at the current positions in CSR form, original ids, ascending in each
 * row, i != j, r^2 < (k h)^2 in the mode's precision (the same test the pair loops use).
 * offsets: n_total + 1 host int64. idx: host int32 of capacity *nnz (in), or NULL to ask
 * only for the size. *nnz receives the count. Debug / parity path, not a fast path. */
sph_status sph_get_neighbors(sph_ctx* ctx, int64_t* offsets, int32_t* idx, int64_t* nnz);

/* One right-hand-side evaluation at the current state without updating it (the
 * SPHEvaluator use of Sec. 3.4). Rates are then readable with sph_get ("arho", "ax",
 * "ay", "az", "xsx", "xsy", "xsz"); with summation density "rho" receives the sum. */
sph_status sph_eval_rhs(sph_ctx* ctx, const sph_scheme* scheme);

/* Advance nsteps predictor-corrector steps (Sec. 2.1, kick-drift-kick for u and x; the
 * density advanced like the positions, rho^{n+1} = rho^n + dt D(x^{n+1}, u^{n+1/2}), then
 * the momentum evaluated at (x^{n+1}, u^{n+1/2}, rho^{n+1}); neighbours rebuilt every
 * step). dt > 0 fixes the
 * step; dt <= 0 takes min(0.25 h / (c0 + max|u|), 0.25 sqrt(h / max|a|), 0.125 h^2 / nu)
 * from the previous evaluation. Rates carried between calls are recomputed first when the
 * state was set or the scheme differs. The steps run as replays of a captured CUDA graph.
 * SPH_ERR_NONFINITE: the state is that of the step where NaN/Inf appeared. */
sph_status sph_step(sph_ctx* ctx, const sph_scheme* scheme, double dt, int32_t nsteps);

/* As sph_step, but returns once the steps are enqueued on the context stream without
 * waiting for them (an initial evaluation, when needed, is enqueued too). Device-side
 * failures (SPH_ERR_NONFINITE) are reported by the next sph_synchronize. */
sph_status sph_step_async(sph_ctx* ctx, const sph_scheme* scheme, double dt, int32_t nsteps);

/* Wait for all work enqueued on the context stream; returns the device status. */
sph_status sph_synchronize(sph_ctx* ctx);

/* Phase timing. enable != 0: steps captured from now on record CUDA events between their
 * phases (a few microseconds of overhead per step). sph_phase_times then gives the device
 * time in ms of the last completed step's phases: out[0] drift + cell keys, out[1] radix
 * sort, out[2] reorder + EOS, out[3] cell table, out[4] density pass (neighbour scan and
 * list, summation density or continuity, EOS), out[5] momentum pass with the corrector
 * kick and the reductions; with SPH_INTEGRATOR_PEC those of the end-of-step build and
 * evaluation. SPH_ERR_STATE if no timed step ran. */
sph_status sph_set_timing(sph_ctx* ctx, int32_t enable);
sph_status sph_phase_times(sph_ctx* ctx, float out[6]);

/* Tile shape of the pair passes: lanes per destination particle (1, 2, 4 or 8) that
 * share its stencil scan (density pass) and its neighbour list (both passes). More lanes
 * hide latency and spread small problems over more SMs. The neighbour list is the same for
 * every shape; the summation order changes (results stay within rounding of each other).
 * Forces a new graph capture. */
sph_status sph_set_groups(sph_ctx* ctx, int32_t momentum_lanes);

/* How a step runs. SPH_STEP_GRAPH (default): the phases (drift + keys, radix sort passes,
 * reorder, cell table, density pass, momentum pass, reductions) as separate kernels in a
 * captured CUDA graph. SPH_STEP_PERSISTENT: the whole step (with the solid-wall pressure
 * phase where the scheme asks for it) as ONE cooperative launch whose blocks stay resident
 * and meet at grid-wide barriers between the phases, captured in a CUDA graph per parity
 * of the state buffers (no launch gaps). Both run the same per-particle code, so the
 * states are equal bitwise; the diagnostics are summed in another order. Steps of the
 * midpoint integrator run as the graph in either mode. SPH_ERR_INVALID if the mode is
 * unknown or the device cannot launch cooperatively. */
enum { SPH_STEP_GRAPH = 0, SPH_STEP_PERSISTENT = 1 };
sph_status sph_set_step_mode(sph_ctx* ctx, int32_t mode);

/* Current tuning: momentum-pass lanes per destination, step mode and density-pass lanes per
 * destination (any may be NULL). */
sph_status sph_get_tuning(const sph_ctx* ctx, int32_t* momentum_lanes, int32_t* mode,
                          int32_t* density_lanes);

/* Time limit of one device-side wait (a grid barrier of the persistent step), in ns;
 * default 1 s; 0 lets no block wait (a persistent step of more than one block then fails
 * at its first barrier). A wait that runs out raises SPH_ERR_TIMEOUT at the next
 * synchronising call; the step is then incomplete and the state must be set again
 * (sph_load_state / sph_set) before stepping on. */
sph_status sph_set_wait_limit(sph_ctx* ctx, uint64_t ns);

/* Autotuner: times each pair pass for every tile shape on the current state (the passes
 * act like sph_eval_rhs) and keeps the fastest shape per pass; then times a few steps in
 * each step mode from the same state, keeps the faster mode and puts the state, time and
 * records back bitwise. Caches the choice for this (precision, dim, kernel, log2 n) for
 * contexts created later in the process and returns the momentum-pass lanes in *chosen
 * (may be NULL). Contexts start from a cached choice, else 4 lanes below 200,000 particles
 * and 1 above, in graph mode. The persistent step uses the momentum-pass shape for both
 * passes. Timing-dependent: call it explicitly, not inside a run whose bitwise
 * reproducibility matters. A batch needs one sph_step_batch call first. */
sph_status sph_autotune(sph_ctx* ctx, const sph_scheme* scheme, int32_t* chosen);

/* Kernel launches one step issues (for launch accounting). */
sph_status sph_kernels_per_step(const sph_ctx* ctx, const sph_scheme* scheme, int32_t* count);

/* Hand-written adjoint of K predictor-corrector steps with fixed dt (the neighbour set of
 * every step held fixed): starting from the current state, runs K steps (the context ends
 * in the final state, as after sph_step) and returns the gradient of the final kinetic
 * energy KE = 1/2 sum_fluid m |u|^2 with respect to
 *   dKE_du0   (host, dim arrays of n_total doubles, original order, walls 0): the fluid
 *             velocities of the current state, which are treated as initial values, with
 *             the initial evaluation recomputed from them (as sph_eval_rhs does);
 *   dKE_dnu   the laminar viscosity nu of the scheme;
 *   dKE_dalpha the artificial-viscosity coefficient alpha (0 when alpha is 0: the term
 *             is then switched off).
 * Any output may be NULL. Checkpoint and recompute: the state is saved every ckpt_every
 * steps (<= 0: ceil(sqrt K)), the segments aligned to the end (the first one holds the
 * remainder); the last segment is taped as the K steps run, every other segment is
 * recomputed once from its checkpoint, taping the pair-loop inputs and the neighbour list
 * of its steps, and each is reversed over the taped lists. Pair
 * terms in the pair-loop precision with compensated sums; adjoint state and the scalar
 * gradients in FP64. Continuity formulation only (SPH_ERR_INVALID for summation density),
 * dt > 0 required. Device workspace: about (K / ckpt_every + 1) * 124 +
 * (ckpt_every + 1) * (48 + 4 * maxn) + 300 bytes per particle in FP32 mode, maxn being the
 * neighbour-list capacity (about twice the largest neighbour count), allocated for the
 * call. */
sph_status sph_backward(sph_ctx* ctx, const sph_scheme* scheme, double dt, int32_t K,
                        int32_t ckpt_every, double* dKE_du0, double* dKE_dnu, double* dKE_dalpha);

/* ---------------------------------------------------------------------------------
 * Batches: many independent problems of uneven size advanced together in the same
 * launches (one CUDA graph per step for all of them). Instances share dim, kernel and
 * precision; each has its own domain (grid), scheme and time step.
 *
 * sph_create_batch: domains[k] and arrays_per_instance[k] consecutive entries of `arrays`
 * describe instance k. Global particle ids (and array indices for sph_get / sph_set)
 * follow the concatenation of all arrays. Other arguments as in sph_create. */
sph_status sph_create_batch(const sph_domain* domains, const sph_array_desc* arrays,
                            const int32_t* arrays_per_instance, int32_t n_instances, void* stream,
                            sph_alloc_fn alloc, sph_free_fn free_fn, void* alloc_user,
                            sph_ctx** out);

/* Advance every instance nsteps steps; schemes[k] and dt[k] (dt <= 0: CFL-type step of
 * that instance) per instance; all instances share the density formulation and the
 * integrator (SPH_ERR_INVALID otherwise). The first
 * call (or a change of schemes or dts) evaluates every instance at its current state.
 * Same integrator and equations as sph_step. Single-problem calls (sph_step,
 * sph_eval_rhs, sph_backward, sph_get_cells, sph_get_neighbors, sph_build_neighbors)
 * return SPH_ERR_STATE on a batch; sph_get, sph_set, sph_set_groups, sph_autotune (scheme
 * ignored, after a first sph_step_batch), sph_set_timing and sph_phase_times work. */
sph_status sph_step_batch(sph_ctx* ctx, const sph_scheme* schemes, const double* dt, int32_t nsteps);

/* As sph_step_batch without waiting for the steps (errors raised on the device are
 * reported by the next sph_synchronize). */
sph_status sph_step_batch_async(sph_ctx* ctx, const sph_scheme* schemes, const double* dt,
                                int32_t nsteps);

/* Diagnostics record (SPH_DIAG_COUNT doubles) of every instance after its last evaluation,
 * instance-major, into out (n_instances * SPH_DIAG_COUNT doubles, host). */
sph_status sph_batch_diagnostics(sph_ctx* ctx, double* out);

/* Property of one array (or -1 for all particles) into a host buffer, original order.
 * prop: "x" "y" "z" "u" "v" "w" "rho" "m", the EDAC pressure "p" (zero unless set or
 * evolved by SPH_DENSITY_EDAC), or rates of the last evaluation "arho" (the pressure rate
 * under SPH_DENSITY_EDAC) "ax" "ay" "az" "xsx" "xsy" "xsz". */
sph_status sph_get(sph_ctx* ctx, int32_t array, const char* prop, double* out);

/* Overwrite one property ("x" "y" "z" "u" "v" "w" "rho" "m" "p") of one array (or -1 for all
 * particles) from a host buffer in original order. Invalidates rates and neighbours. */
sph_status sph_set(sph_ctx* ctx, int32_t array, const char* prop, const double* in);

/* Diagnostics record of the last evaluation (SPH_DIAG_COUNT doubles, host). */
sph_status sph_diagnostics(sph_ctx* ctx, double* out);

/* Records of the steps of the last sph_step call, oldest first, into out
 * (capacity max_records * SPH_DIAG_COUNT doubles); *count receives how many were written.
 * The context keeps the most recent 65536 records. */
sph_status sph_history(sph_ctx* ctx, double* out, int32_t max_records, int32_t* count);

/* Full device state (positions, velocities, density, mass, EDAC pressure, rates, internal
 * order, time)
 * to/from a host buffer. buf NULL: *bytes receives the size. Loading restores the exact
 * state so that a resumed run is bitwise identical to an uninterrupted one. */
sph_status sph_save_state(sph_ctx* ctx, void* buf, size_t* bytes);
sph_status sph_load_state(sph_ctx* ctx, const void* buf, size_t bytes);

/* As sph_save_state / sph_load_state (the output and restart of Sec. 3.3), but the copies
 * are only enqueued on the context stream, behind the work already there: the call returns
 * at once, and the buffer must stay valid (for a load: unchanged; for a save: unread) until
 * sph_synchronize returns. In a pinned host buffer the copies run on the copy engines while
 * other contexts compute, so a run that streams states through several contexts overlaps
 * its transfers with its steps. Errors of the enqueued copies are reported by
 * sph_synchronize; argument errors as by the synchronous calls. */
sph_status sph_save_state_async(sph_ctx* ctx, void* buf, size_t* bytes);
sph_status sph_load_state_async(sph_ctx* ctx, const void* buf, size_t bytes);

/* ---------------------------------------------------------------------------------
 * Allocation-free cell sort. The paper has no counterpart: this entry point exists for
 * callers that cannot allocate device memory -- for example code that runs inside a
 * host framework whose memory pool has already reserved the device (any cudaMalloc
 * beyond that budget fails or is forbidden), or a latency-critical loop where
 * cudaMalloc's implicit device-wide synchronisation is not acceptable. It performs the
 * neighbour-build sort of sph_build_neighbors on caller-owned device buffers and calls
 * no cudaMalloc, cudaFree or other allocating routine.
 *
 * Scratch: one fixed device array of about 12.8 MB inside the library (keys, values and
 * histograms for up to SPH_NOALLOC_MAX_PARTICLES particles). Every GPU that loads the
 * library holds it until the process exits. All calls share it and it keeps the last
 * call's contents: calls whose work overlaps on the GPU (for example on two streams, or
 * from two threads) race on it and must be serialised by the caller.
 *
 * Set-up: the first call on each device looks up that device's address of the array
 * (cudaGetSymbolAddress, with the device current) and keeps it for later calls; make that
 * first call before any stream capture on the device. Each later call checks the kept
 * address (cudaPointerGetAttributes) and looks it up again when a device reset has
 * unloaded the array.
 *
 *  domain        grid and binning as in sph_create (dim, kernel, precision, periodic, h,
 *                lo, hi); the cell count follows the same rule.
 *  x, y, z       device pointers to n FP64 positions (z NULL in 2D). Positions on a
 *                periodic axis must already lie in [lo, hi); positions outside the box
 *                are clamped into the edge cells.
 *  n             particle count, 0 <= n <= SPH_NOALLOC_MAX_PARTICLES; larger n returns
 *                SPH_ERR_CAPACITY before any device work.
 *  order         device, n entries (out): input index at each sorted position; a stable
 *                sort by linear cell id, so ties keep the input order.
 *  cell_offsets  device, offsets_capacity entries (out): offsets[c] = number of particles
 *                in cells < c, ncells + 1 entries. NULL: only *ncells_out is set.
 *  ncells_out    host (out): number of cells.
 *  stream        cudaStream_t the work is enqueued on (NULL: legacy default stream); the
 *                call returns without waiting for it.
 * Errors: SPH_ERR_INVALID (bad domain or NULL buffer), SPH_ERR_CAPACITY (n too large or
 * offsets_capacity < ncells + 1), SPH_ERR_CUDA; the message is in sph_last_error(NULL). */
#define SPH_NOALLOC_MAX_PARTICLES 1048576
sph_status sph_cell_sort_noalloc(const sph_domain* domain, const double* x, const double* y,
                                 const double* z, int64_t n, uint32_t* order,
                                 uint32_t* cell_offsets, int64_t offsets_capacity,
                                 int64_t* ncells_out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SPH_H */
