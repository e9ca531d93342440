/*
 * C ABI of the neighbour search with a per-particle smoothing length (the variable-support
 * case of Sec. 2.2 of the PySPH paper, which the paper answers with an octree: split a node
 * into its octants while it holds more than a given number of particles, descend at query
 * time only into the nodes that can hold a neighbour).
 *
 * Relation: particle i carries its own smoothing length h_i; j != i is a neighbour of i
 * when |x_i - x_j| < k max(h_i, h_j) (k = 3 for the quintic spline, 2 for the Wendland C2
 * and the cubic spline), the squared distance ((dx dx) + dy dy) + dz dz and the radius
 * k max(h_i, h_j) rounded op by op in the precision of the mode from the positions and h
 * rounded to it. The relation is symmetric; no periodic axes. The same pass computes the
 * summation density (Eq. 2) with the pair smoothing length h_ij = (h_i + h_j) / 2:
 *   rho_i = m_i W(0, h_i) + sum_{j neighbour of i} m_j W(|x_i - x_j|, h_ij),
 * in FP64 (SPH_PREC_FP64) or in FP32 with compensated sums (SPH_PREC_FP32).
 *
 * Ownership: the context owns all device memory (through the allocator callbacks when
 * given, else cudaMalloc) and copies the inputs in; outputs go to caller buffers. Every
 * call returns a status and sets a message (sph_vh_last_error); nothing aborts. A context
 * is used from one thread at a time. All work runs on the context's stream.
 */
#ifndef SPH_VH_H
#define SPH_VH_H

#include "sph.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sph_vh sph_vh;

typedef struct {
    int32_t dim;        /* 2 or 3 */
    int32_t kernel;     /* SPH_KERNEL_QUINTIC, SPH_KERNEL_WENDLAND_C2, SPH_KERNEL_CUBIC_SPLINE */
    int32_t precision;  /* SPH_PREC_FP64 or SPH_PREC_FP32: the predicate, boxes and sums */
    int32_t leaf_size;  /* a node with more particles than this splits (1 .. 4096) */
} sph_vh_params;

/* A context for up to `capacity` particles (>= 0). stream: a cudaStream_t or NULL (a stream
 * of its own). alloc / free_fn: device allocator callbacks (both or neither). */
sph_status sph_vh_create(const sph_vh_params* params, int64_t capacity, void* stream,
                         sph_alloc_fn alloc, sph_free_fn free_fn, void* alloc_user, sph_vh** out);

/* Particles (host arrays of n FP64 values, copied to the device; z ignored in 2D and may
 * then be NULL): positions, smoothing lengths (> 0, finite) and masses.
 * SPH_ERR_INVALID if n exceeds the capacity or an h is not positive and finite. */
sph_status sph_vh_set(sph_vh* ctx, int64_t n, const double* x, const double* y, const double* z,
                      const double* h, const double* m);

/* The search on the particles last set: root box, keys, sort, tree, then the neighbour
 * lists and the density. Waits for the stream. The list slots per particle grow to the
 * largest count seen (the first search, or one whose counts grew, runs the query twice).
 * SPH_ERR_STATE before sph_vh_set; SPH_ERR_TIMEOUT if a device wait ran out. */
sph_status sph_vh_search(sph_vh* ctx);

/* Neighbour lists in CSR form in the caller's particle order (host buffers): offsets[n + 1]
 * and, when idx is not NULL, idx[nnz] (particle indices; inside a row in the order the
 * walk met them, not sorted). *nnz gets the total. SPH_ERR_CAPACITY if idx_capacity < nnz
 * (offsets and *nnz are still written). */
sph_status sph_vh_neighbors(sph_vh* ctx, int64_t* offsets, int32_t* idx, int64_t idx_capacity,
                            int64_t* nnz);

/* Density of the last search, host array of n FP64 values in the caller's order. */
sph_status sph_vh_density(sph_vh* ctx, double* rho);

/* Figures of the last search: out[0] nodes, out[1] leaves, out[2] deepest level with nodes,
 * out[3] pairs examined in the leaves, out[4] neighbour pairs (ordered), out[5] largest
 * neighbour count, out[6] list slots per particle, out[7] query launches of the search. */
sph_status sph_vh_stats(sph_vh* ctx, int64_t out[8]);

/* The tree of the last search, for checks (host buffers, NULL to skip): per node
 * start / end (range in key order), child (first child node or -1) and nchild, lo[3 * nodes]
 * and hi[3 * nodes] (box, FP64 of the mode values), hmax[nodes]; perm[n]: the caller's
 * index of each key-order position. nodes_capacity: entries of the node buffers
 * (SPH_ERR_CAPACITY if smaller than out[0] of sph_vh_stats). */
sph_status sph_vh_tree(sph_vh* ctx, int64_t nodes_capacity, int32_t* start, int32_t* end,
                       int32_t* child, int32_t* nchild, double* lo, double* hi, double* hmax,
                       int32_t* perm);

/* Timing of the searches (off by default): with enable, each search records CUDA events
 * around its two phases; sph_vh_phase_times gives, for the last search, out[0] = ms from
 * the start to the built tree (root box, keys, sort, gather, levels, boxes) and out[1] =
 * ms of the query (walk, lists, density). SPH_ERR_STATE if the last search was not timed
 * or had no particles. */
sph_status sph_vh_set_timing(sph_vh* ctx, int32_t enable);
sph_status sph_vh_phase_times(sph_vh* ctx, float out[2]);

/* Message of the last failed call on ctx (or of the last failed sph_vh_create if NULL). */
const char* sph_vh_last_error(const sph_vh* ctx);

void sph_vh_destroy(sph_vh* ctx);

#ifdef __cplusplus
}
#endif

#endif /* SPH_VH_H */
