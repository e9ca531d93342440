// Neighbour search with a per-particle smoothing length through an octree (Sec. 2.2: a
// uniform grid needs cells of the largest support radius when the radius varies, so the
// paper searches such particle sets with an octree that splits a node into its 8 octants
// (4 quadrants in 2D) while it holds more than a given number of particles, and answers a
// query by descending only into the nodes that can hold a neighbour).
//
// Relation (reading C-VH): j != i is a neighbour of i when |x_i - x_j| < k max(h_i, h_j),
// r^2 = ((dx dx) + dy dy) + dz dz and R = k max(h_i, h_j) rounded op by op in the mode's
// precision from the positions and h rounded to it (no fused multiply-add), no periodic
// axes. The summation density of the same pass takes the pair smoothing length
// h_ij = (h_i + h_j) / 2: rho_i = m_i W(0, h_i) + sum_j m_j W(r_ij, h_ij) (Eq. 2).
//
// GB300 design:
//  - keys: Morton codes of the positions quantised to 2^B cells per axis of the root cube
//    (B = 10 in 3D, 15 in 2D: 30-bit keys), sorted by the library's one-sweep radix sort
//    (4 passes); the particle data are then gathered once into key order, so every node is
//    a contiguous range and a leaf's particles are one run of 16- or 32-byte records;
//  - the tree is built top-down, one launch per level: a node with more than leaf_size
//    particles finds its children's ranges by binary search on the next key digit and
//    takes slots for its non-empty children from the level's counter (the slot numbers
//    depend on scheduling, the tree's shape and every traversal order do not);
//  - node boxes and the largest h are set bottom-up, one launch per level, from the
//    particles' mode-precision records, so the pruning test is exact: the box distance is
//    formed with the same rounded operations as a pair distance and is never larger than
//    the distance to any particle inside, so a node that holds a neighbour is never
//    skipped (no margin needed);
//  - the query is a depth-first walk per particle in key order, done by a warp for 32
//    neighbouring particles at once (the warp enters a node any of them needs, so control
//    flow is uniform), with an explicit stack and staged leaf records in shared memory,
//    writing the neighbour list interleaved (nl[k * n + i], coalesced for the warp) and the
//    density in one pass.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "sph_device.cuh"
#include "sph_launch.h"
#include "sort_impl.cuh"
#include "sph_vh.h"

namespace sph {

constexpr int VH_THREADS = 256;
constexpr int VH_STACK = 80;      // >= (2^d - 1) B + 1 entries of a depth-first walk
constexpr int VH_LEVELS = 16;     // levels 0..B (B <= 15)
constexpr int VH_PASSES = 4;      // 30-bit keys, 8-bit digits

__host__ __device__ constexpr int vh_bits(int dim) { return dim == 3 ? 10 : 15; }

// A node: tight box of its particles and their largest h (mode precision), its range in
// key order, and its children (contiguous slots; child < 0: a leaf).
template <class Real>
struct VhNode {
    typename V4<Real>::T lo;  // lo.x lo.y lo.z, lo.w = largest h
    typename V4<Real>::T hi;  // hi.x hi.y hi.z
    int4 r;                   // start, end, child, nchild
};

// Device bookkeeping of one search.
struct VhDev {
    double lo[3];            // root cube corner
    double inv_cell;         // 2^B / side
    uint32_t level_n[VH_LEVELS + 1];  // nodes per level (level_n[0] = 1: the root)
    unsigned long long cand, pairs;   // pairs examined, neighbours found
    uint32_t max_count;      // largest neighbour count of a particle
    uint32_t leaves;
};

// Exact FP operations (no contraction into fused multiply-adds), as the predicate of the
// reading prescribes.
__device__ __forceinline__ float vh_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float vh_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float vh_sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double vh_mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double vh_add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double vh_sub(double a, double b) { return __dsub_rn(a, b); }

// ------------------------------------------------------------------ root box
// Stage 1: per-block min / max of the positions (FP64) into part[block][6].
__global__ void __launch_bounds__(VH_THREADS)
k_vh_bounds(const double* __restrict__ x, const double* __restrict__ y,
            const double* __restrict__ z, int n, int dim, double* __restrict__ part) {
    double v[6] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY};
    const double* xs[3] = {x, y, z};
    for (int i = blockIdx.x * VH_THREADS + threadIdx.x; i < n; i += gridDim.x * VH_THREADS)
        for (int d = 0; d < dim; ++d) {
            const double a = xs[d][i];
            v[d] = fmin(v[d], a);
            v[3 + d] = fmax(v[3 + d], a);
        }
    __shared__ double red[VH_THREADS / 32][6];
    for (int q = 0; q < 6; ++q)
        for (int o = 16; o > 0; o >>= 1) {
            const double t = __shfl_down_sync(0xffffffffu, v[q], o);
            v[q] = q < 3 ? fmin(v[q], t) : fmax(v[q], t);
        }
    if ((threadIdx.x & 31) == 0)
        for (int q = 0; q < 6; ++q) red[threadIdx.x >> 5][q] = v[q];
    __syncthreads();
    if (threadIdx.x < 6) {
        double t = red[0][threadIdx.x];
        for (int w = 1; w < VH_THREADS / 32; ++w)
            t = threadIdx.x < 3 ? fmin(t, red[w][threadIdx.x]) : fmax(t, red[w][threadIdx.x]);
        part[blockIdx.x * 6 + threadIdx.x] = t;
    }
}

// Stage 2 (one warp): the root cube, its quantisation scale and the level counters.
__global__ void k_vh_root(const double* __restrict__ part, int nblocks, int dim, int n, VhDev* dev) {
    const int lane = threadIdx.x;
    double v[6] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY};
    for (int b = lane; b < nblocks; b += 32)
        for (int q = 0; q < 6; ++q)
            v[q] = q < 3 ? fmin(v[q], part[b * 6 + q]) : fmax(v[q], part[b * 6 + q]);
    for (int q = 0; q < 6; ++q)
        for (int o = 16; o > 0; o >>= 1) {
            const double t = __shfl_down_sync(0xffffffffu, v[q], o);
            v[q] = q < 3 ? fmin(v[q], t) : fmax(v[q], t);
        }
    if (lane == 0) {
        double side = 0.0;
        for (int d = 0; d < 3; ++d) {
            const double lo = d < dim && n > 0 ? v[d] : 0.0;
            const double hi = d < dim && n > 0 ? v[3 + d] : 0.0;
            dev->lo[d] = lo;
            side = fmax(side, hi - lo);
        }
        side = side > 0.0 ? side * (1.0 + 1e-12) : 1.0;  // the largest coordinate stays inside
        dev->inv_cell = (double)(1 << vh_bits(dim)) / side;
        for (int l = 0; l <= VH_LEVELS; ++l) dev->level_n[l] = 0u;
        dev->level_n[0] = n > 0 ? 1u : 0u;
        dev->cand = 0ull;
        dev->pairs = 0ull;
        dev->max_count = 0u;
        dev->leaves = 0u;
    }
}

// ---------------------------------------------------------------- Morton keys
__device__ __forceinline__ uint32_t vh_spread3(uint32_t v) {  // 10 bits -> every third bit
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}
__device__ __forceinline__ uint32_t vh_spread2(uint32_t v) {  // 15 bits -> every second bit
    v &= 0x7fffu;
    v = (v | (v << 8)) & 0x00ff00ffu;
    v = (v | (v << 4)) & 0x0f0f0f0fu;
    v = (v | (v << 2)) & 0x33333333u;
    v = (v | (v << 1)) & 0x55555555u;
    return v;
}

// Keys (x in the lowest bit of each digit) and the digit histograms of all sort passes.
template <int DIM>
__global__ void __launch_bounds__(VH_THREADS)
k_vh_keys(const double* __restrict__ x, const double* __restrict__ y, const double* __restrict__ z,
          int n, const VhDev* __restrict__ dev, uint32_t* __restrict__ keys, uint32_t* __restrict__ ghist) {
    __shared__ uint32_t h[VH_PASSES][RADIX];
    for (int p = 0; p < VH_PASSES; ++p) h[p][threadIdx.x] = 0u;
    __syncthreads();
    constexpr uint32_t top = (1u << vh_bits(DIM)) - 1u;
    const double* xs[3] = {x, y, z};
    for (int base = blockIdx.x * VH_THREADS; base < n; base += gridDim.x * VH_THREADS) {
        const int i = base + threadIdx.x;
        const bool valid = i < n;
        uint32_t key = 0u;
        if (valid) {
            uint32_t c[3] = {0u, 0u, 0u};
            for (int d = 0; d < DIM; ++d) {
                const double v = floor((xs[d][i] - dev->lo[d]) * dev->inv_cell);
                c[d] = v > 0.0 ? (v < (double)top ? (uint32_t)v : top) : 0u;
            }
            key = DIM == 3 ? (vh_spread3(c[0]) | (vh_spread3(c[1]) << 1) | (vh_spread3(c[2]) << 2))
                           : (vh_spread2(c[0]) | (vh_spread2(c[1]) << 1));
            keys[i] = key;
        }
        digit_hist_add(key, valid, VH_PASSES, h);
    }
    __syncthreads();
    for (int p = 0; p < VH_PASSES; ++p) {
        const uint32_t v = h[p][threadIdx.x];
        if (v) atomicAdd(&ghist[p * RADIX + threadIdx.x], v);
    }
}

// Gather into key order: the mode-precision records P = (x, y, z, h) and the masses; the
// root node's range.
template <class Real>
__global__ void __launch_bounds__(VH_THREADS)
k_vh_gather(const double* __restrict__ x, const double* __restrict__ y, const double* __restrict__ z,
            const double* __restrict__ h, const double* __restrict__ m, const uint32_t* __restrict__ perm,
            int n, int dim, typename V4<Real>::T* __restrict__ P, Real* __restrict__ M,
            VhNode<Real>* __restrict__ nodes) {
    for (int k = blockIdx.x * VH_THREADS + threadIdx.x; k < n; k += gridDim.x * VH_THREADS) {
        const uint32_t o = perm[k];
        typename V4<Real>::T p;
        p.x = (Real)x[o];
        p.y = (Real)y[o];
        p.z = dim == 3 ? (Real)z[o] : Real(0);
        p.w = (Real)h[o];
        P[k] = p;
        M[k] = (Real)m[o];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) nodes[0].r = make_int4(0, n, -1, 0);
}

// ------------------------------------------------------------------ the tree
__device__ __forceinline__ uint32_t vh_level_begin(const VhDev* dev, int level) {
    uint32_t b = 0u;
    for (int l = 0; l < level; ++l) b += dev->level_n[l];
    return b;
}

// Nodes of a level that exist (slots past the capacity were never written).
__device__ __forceinline__ uint32_t vh_level_count(const VhDev* dev, int level, uint32_t begin,
                                                   uint32_t node_cap) {
    const uint32_t c = dev->level_n[level];
    return begin >= node_cap ? 0u : (c < node_cap - begin ? c : node_cap - begin);
}

// Level `level`: every node with more than leaf particles (and a level below B) takes slots
// for its non-empty children at level + 1 and writes their ranges.
template <class Real, int DIM>
__global__ void __launch_bounds__(VH_THREADS)
k_vh_split(VhNode<Real>* __restrict__ nodes, VhDev* dev, int level, const uint32_t* __restrict__ keys,
           int leaf, uint32_t node_cap, Control* ctl) {
    constexpr int B = vh_bits(DIM), NCH = 1 << DIM;
    const uint32_t begin = vh_level_begin(dev, level);
    const uint32_t count = vh_level_count(dev, level, begin, node_cap);
    const uint32_t next_begin = begin + dev->level_n[level];
    const int shift = DIM * (B - level - 1);
    for (uint32_t t = blockIdx.x * VH_THREADS + threadIdx.x; t < count; t += gridDim.x * VH_THREADS) {
        const uint32_t node = begin + t;
        int4 r = nodes[node].r;
        const int s = r.x, e = r.y;
        if (e - s <= leaf || level >= B) {
            r.z = -1;
            r.w = 0;
            nodes[node].r = r;
            continue;
        }
        // bnd[o] = first particle of the range whose digit at this level is >= o (the digits
        // do not decrease inside a node: the keys are sorted and share the node's prefix)
        int bnd[NCH + 1];
        bnd[0] = s;
        bnd[NCH] = e;
        for (int o = 1; o < NCH; ++o) {
            int lo = bnd[o - 1], hi = e;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if ((int)((keys[mid] >> shift) & (NCH - 1)) < o) lo = mid + 1;
                else hi = mid;
            }
            bnd[o] = lo;
        }
        int c = 0;
        for (int o = 0; o < NCH; ++o) c += bnd[o + 1] > bnd[o] ? 1 : 0;
        const uint32_t slot = next_begin + atomicAdd(&dev->level_n[level + 1], (uint32_t)c);
        if (slot + (uint32_t)c > node_cap) {
            // no room (the capacity bound of the context makes this unreachable): the node
            // stays a leaf and the slots it took that exist become empty leaves, which no
            // query enters (their box is empty)
            atomicOr(&ctl->status, ST_CAPACITY);
            for (uint32_t q = slot; q < slot + (uint32_t)c && q < node_cap; ++q)
                nodes[q].r = make_int4(0, 0, -1, 0);
            r.z = -1;
            r.w = 0;
            nodes[node].r = r;
            continue;
        }
        int w = 0;
        for (int o = 0; o < NCH; ++o)
            if (bnd[o + 1] > bnd[o]) nodes[slot + w++].r = make_int4(bnd[o], bnd[o + 1], -1, 0);
        r.z = (int)slot;
        r.w = c;
        nodes[node].r = r;
    }
}

// Level `level`, deepest first: a leaf's tight box and largest h from its particles, an
// inner node's from its children.
template <class Real>
__global__ void __launch_bounds__(VH_THREADS)
k_vh_boxes(VhNode<Real>* __restrict__ nodes, VhDev* dev, int level,
           const typename V4<Real>::T* __restrict__ P, uint32_t node_cap) {
    using V = typename V4<Real>::T;
    const uint32_t begin = vh_level_begin(dev, level);
    const uint32_t count = vh_level_count(dev, level, begin, node_cap);
    uint32_t leaves = 0u;
    for (uint32_t t = blockIdx.x * VH_THREADS + threadIdx.x; t < count; t += gridDim.x * VH_THREADS) {
        const uint32_t node = begin + t;
        const int4 r = nodes[node].r;
        V lo, hi;
        lo.x = lo.y = lo.z = lo.w = (Real)INFINITY;
        hi.x = hi.y = hi.z = (Real)-INFINITY;
        hi.w = Real(0);
        lo.w = Real(0);
        if (r.z < 0) {
            ++leaves;
            for (int k = r.x; k < r.y; ++k) {
                const V p = P[k];
                lo.x = fmin(lo.x, p.x); lo.y = fmin(lo.y, p.y); lo.z = fmin(lo.z, p.z);
                hi.x = fmax(hi.x, p.x); hi.y = fmax(hi.y, p.y); hi.z = fmax(hi.z, p.z);
                lo.w = fmax(lo.w, p.w);
            }
        } else {
            for (int c = r.z; c < r.z + r.w; ++c) {
                const V a = nodes[c].lo, b = nodes[c].hi;
                lo.x = fmin(lo.x, a.x); lo.y = fmin(lo.y, a.y); lo.z = fmin(lo.z, a.z);
                hi.x = fmax(hi.x, b.x); hi.y = fmax(hi.y, b.y); hi.z = fmax(hi.z, b.z);
                lo.w = fmax(lo.w, a.w);
            }
        }
        nodes[node].lo = lo;
        nodes[node].hi = hi;
    }
    for (int o = 16; o > 0; o >>= 1) leaves += __shfl_down_sync(0xffffffffu, leaves, o);
    if ((threadIdx.x & 31) == 0 && leaves) atomicAdd(&dev->leaves, leaves);
}

// ------------------------------------------------------------------ the query
// Normalisation of the unscaled smoothing functions of sph_device.cuh (the cubic spline
// there is four times the M4 B-spline).
__host__ __device__ inline double vh_sigma(int kernel, int dim) {
    const double pi = 3.14159265358979323846;
    if (kernel == QUINTIC) return dim == 2 ? 7.0 / (478.0 * pi) : 1.0 / (120.0 * pi);
    if (kernel == CUBIC_SPLINE) return dim == 2 ? 5.0 / (14.0 * pi) : 1.0 / (4.0 * pi);
    return dim == 2 ? 7.0 / (4.0 * pi) : 21.0 / (16.0 * pi);
}

// The query: a depth-first walk from the root for particle i of the key order that enters
// a node when the box distance is below k max(h_i, largest h in the node), and tests every
// particle of an entered leaf with the exact predicate. A warp walks together for 32
// consecutive particles (spatially close, so their walks nearly coincide): it enters a node
// when any of its particles needs it (ballot), so control flow is uniform; the stack lives
// in shared memory and a leaf's records are staged there 32 at a time, read back by every
// lane as a broadcast. A particle tests only the leaves it needs itself. Writes the
// neighbours (key-order indices, in walk order) to nl[k * n + i] for k < maxn, the count
// to cnt[i] (the true count also when it exceeds maxn, which raises ST_CAPACITY), and
// rho[i] (FP64, caller order through perm). Measured on 10^6 particles of the Gaussian
// blob, 3D, leaves of 16: 2.03 ms, against 3.36 ms when each thread walked alone.
template <class Real, int DIM, int KERNEL>
__global__ void __launch_bounds__(VH_THREADS)
k_vh_query_warp(const typename V4<Real>::T* __restrict__ P, const Real* __restrict__ M,
                const VhNode<Real>* __restrict__ nodes, int n, uint32_t* __restrict__ nl,
                uint32_t* __restrict__ cnt, int maxn, double* __restrict__ rho,
                const uint32_t* __restrict__ perm, VhDev* dev, Control* ctl) {
    using V = typename V4<Real>::T;
    constexpr int WARPS = VH_THREADS / 32;
    __shared__ int stack_s[WARPS][VH_STACK];
    __shared__ V rec_s[WARPS][32];
    __shared__ Real mass_s[WARPS][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int* stack = stack_s[w];
    V* rec = rec_s[w];
    Real* mass = mass_s[w];
    const Real kf = KERNEL == QUINTIC ? Real(3) : Real(2);
    const Real sigma = (Real)vh_sigma(KERNEL, DIM);
    unsigned long long cand = 0ull, pairs = 0ull;
    uint32_t most = 0u;
    bool overflow = false;
    const int nwarps = (n + 31) / 32;
    for (int wi = blockIdx.x * WARPS + w; wi < nwarps; wi += gridDim.x * WARPS) {
        const int i = wi * 32 + lane;
        const bool valid = i < n;
        V pi;
        pi.x = pi.y = pi.z = pi.w = Real(0);
        if (valid) pi = P[i];
        uint32_t count = 0u;
        Acc<Real> sum;
        sum.zero();
        int sp = 1;
        if (lane == 0) stack[0] = 0;
        __syncwarp();
        while (sp > 0) {
            const int node = stack[--sp];
            const V lo = nodes[node].lo, hi = nodes[node].hi;
            const int4 r = nodes[node].r;
            Real d2 = Real(0);
            {
                const Real c[3] = {pi.x, pi.y, pi.z};
                const Real bl[3] = {lo.x, lo.y, lo.z}, bh[3] = {hi.x, hi.y, hi.z};
#pragma unroll
                for (int d = 0; d < DIM; ++d) {
                    Real e = Real(0);
                    if (c[d] < bl[d]) e = vh_sub(bl[d], c[d]);
                    else if (c[d] > bh[d]) e = vh_sub(c[d], bh[d]);
                    d2 = vh_add(d2, vh_mul(e, e));
                }
            }
            const Real Rn = vh_mul(kf, pi.w > lo.w ? pi.w : lo.w);
            const bool need = valid && d2 < vh_mul(Rn, Rn);
            __syncwarp();  // every lane has read the popped entry
            if (!__any_sync(0xffffffffu, need)) continue;
            if (r.z >= 0) {  // children in reverse, so the first is walked first
                if (sp + r.w > VH_STACK) {
                    overflow = true;  // unreachable for depth <= B (see VH_STACK)
                    continue;
                }
                if (lane < r.w) stack[sp + r.w - 1 - lane] = r.z + lane;
                sp += r.w;
                __syncwarp();
                continue;
            }
            for (int j0 = r.x; j0 < r.y; j0 += 32) {
                const int m = min(32, r.y - j0);
                if (lane < m) {
                    rec[lane] = P[j0 + lane];
                    mass[lane] = M[j0 + lane];
                }
                __syncwarp();
                if (need) {
                    for (int t = 0; t < m; ++t) {
                        const int j = j0 + t;
                        if (j == i) continue;
                        const V pj = rec[t];
                        ++cand;
                        const Real dx = vh_sub(pi.x, pj.x), dy = vh_sub(pi.y, pj.y);
                        Real r2 = vh_add(vh_mul(dx, dx), vh_mul(dy, dy));
                        if (DIM == 3) {
                            const Real dz = vh_sub(pi.z, pj.z);
                            r2 = vh_add(r2, vh_mul(dz, dz));
                        }
                        const Real R = vh_mul(kf, pi.w > pj.w ? pi.w : pj.w);
                        if (!(r2 < vh_mul(R, R))) continue;
                        if ((int)count < maxn) nl[(size_t)count * n + i] = (uint32_t)j;
                        ++count;
                        const Real inv = PairMath<Real>::rcp(Real(0.5) * (pi.w + pj.w));
                        const Real q = PairMath<Real>::sqrt(r2) * inv;
                        Real wn = inv * inv;
                        if (DIM == 3) wn *= inv;
                        if (q < kf) sum.add(mass[t] * (sigma * wn * kernel_w<Real, KERNEL>(q)));
                    }
                }
                __syncwarp();  // the staged records are read before the next ones land
            }
        }
        if (valid) {
            cnt[i] = count;
            pairs += count;
            most = count > most ? count : most;
            if ((int)count > maxn) overflow = true;
            Real w0 = PairMath<Real>::rcp(pi.w);
            Real wn = w0 * w0;
            if (DIM == 3) wn *= w0;
            const double self = (double)M[i] * ((double)sigma * (double)wn * (double)kernel_w<Real, KERNEL>(Real(0)));
            rho[perm[i]] = self + sum.value();
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        cand += __shfl_down_sync(0xffffffffu, cand, o);
        pairs += __shfl_down_sync(0xffffffffu, pairs, o);
        const uint32_t t = __shfl_down_sync(0xffffffffu, most, o);
        most = t > most ? t : most;
    }
    if (lane == 0) {
        atomicAdd(&dev->cand, cand);
        atomicAdd(&dev->pairs, pairs);
        atomicMax(&dev->max_count, most);
    }
    if (overflow) atomicOr(&ctl->status, ST_CAPACITY);
}

}  // namespace sph

// =================================================================== C ABI
using namespace sph;

struct sph_vh {
    sph_vh_params prm{};
    int64_t cap = 0;
    int n = 0;
    bool have = false, searched = false;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    sph_alloc_fn alloc = nullptr;
    sph_free_fn free_fn = nullptr;
    void* user = nullptr;
    std::string err;
    int sms = 1;
    // device memory
    std::vector<void*> blocks;
    double* in[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};  // x y z h m, caller order
    uint32_t* keys[2] = {nullptr, nullptr};
    uint32_t* vals[2] = {nullptr, nullptr};
    uint32_t* work = nullptr;
    size_t work_words = 0;
    void* rec = nullptr;  // key-order records (x, y, z, h) in the mode precision
    void* M = nullptr;
    void* nodes = nullptr;
    uint32_t node_cap = 0;
    VhDev* dev = nullptr;
    Control* ctl = nullptr;
    double* part = nullptr;
    int part_blocks = 0;
    uint32_t* cnt = nullptr;
    double* rho = nullptr;
    uint32_t* nl = nullptr;
    int maxn = 0;
    int sorted = 0;  // buffer index of the sorted keys / permutation
    VhDev host{};    // bookkeeping of the last search
    int query_runs = 0;
    cudaGraphExec_t graph = nullptr;
    int graph_n = -1, graph_maxn = -1;
    bool timing = false, graph_timed = false;
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};  // start, tree built, query done
};

namespace {

thread_local std::string g_vh_error;

sph_status vfail(sph_vh* c, sph_status s, const std::string& msg) {
    if (c) c->err = msg;
    else g_vh_error = msg;
    return s;
}

#define VCK(call)                                                                            \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess) return vfail(c, SPH_ERR_CUDA, std::string(#call ": ") + cudaGetErrorString(e_)); \
    } while (0)

void* vh_alloc(sph_vh* c, size_t bytes) {
    if (bytes == 0) bytes = 16;
    void* p = nullptr;
    if (c->alloc) p = c->alloc(bytes, c->user);
    else if (cudaMalloc(&p, bytes) != cudaSuccess) p = nullptr;
    if (!p) cudaGetLastError();
    return p;
}

void vh_release(sph_vh* c, void* p) {
    if (!p) return;
    if (c->free_fn) c->free_fn(p, c->user);
    else cudaFree(p);
}

void vh_drop_graph(sph_vh* c) {
    if (c->graph) cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
    c->graph_n = c->graph_maxn = -1;
}

int vh_grid(long long n, int cap) {
    long long b = (n + VH_THREADS - 1) / VH_THREADS;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (int)b;
}

template <class Real, int DIM>
void vh_build_t(sph_vh* c) {
    using V = typename V4<Real>::T;
    constexpr int B = vh_bits(DIM);
    const int n = c->n;
    cudaStream_t st = c->stream;
    const int g = vh_grid(n, c->sms * 8);
    k_vh_bounds<<<c->part_blocks, VH_THREADS, 0, st>>>(c->in[0], c->in[1], c->in[2], n, DIM, c->part);
    k_vh_root<<<1, 32, 0, st>>>(c->part, c->part_blocks, DIM, n, c->dev);
    k_vh_keys<DIM><<<g, VH_THREADS, 0, st>>>(c->in[0], c->in[1], c->in[2], n, c->dev, c->keys[0], c->work);
    c->sorted = launch_onesweep(n, c->keys, c->vals, VH_PASSES, c->work, c->ctl, 1000000000ull, st);
    const uint32_t* perm = c->vals[c->sorted];
    k_vh_gather<Real><<<g, VH_THREADS, 0, st>>>(c->in[0], c->in[1], c->in[2], c->in[3], c->in[4], perm, n,
                                               DIM, (V*)c->rec, (Real*)c->M, (VhNode<Real>*)c->nodes);
    const int gs = vh_grid(n, c->sms * 8);
    for (int l = 0; l < B; ++l)
        k_vh_split<Real, DIM><<<gs, VH_THREADS, 0, st>>>((VhNode<Real>*)c->nodes, c->dev, l,
                                                        c->keys[c->sorted], c->prm.leaf_size, c->node_cap,
                                                        c->ctl);
    for (int l = B; l >= 0; --l)
        k_vh_boxes<Real><<<gs, VH_THREADS, 0, st>>>((VhNode<Real>*)c->nodes, c->dev, l, (const V*)c->rec,
                                                   c->node_cap);
}

template <class Real, int DIM, int KERNEL>
void vh_query_t(sph_vh* c) {
    using V = typename V4<Real>::T;
    const int n = c->n;
    const int gq = (int)((n + VH_THREADS - 1) / VH_THREADS);
    k_vh_query_warp<Real, DIM, KERNEL><<<gq < 1 ? 1 : gq, VH_THREADS, 0, c->stream>>>(
        (const V*)c->rec, (const Real*)c->M, (const VhNode<Real>*)c->nodes, n, c->nl, c->cnt, c->maxn,
        c->rho, c->vals[c->sorted], c->dev, c->ctl);
}

template <class Real>
void vh_query_k(sph_vh* c) {
    const int sel = (c->prm.dim == 3 ? 3 : 0) + c->prm.kernel;
    switch (sel) {
        case 0: vh_query_t<Real, 2, QUINTIC>(c); break;
        case 1: vh_query_t<Real, 2, WENDLAND_C2>(c); break;
        case 2: vh_query_t<Real, 2, CUBIC_SPLINE>(c); break;
        case 3: vh_query_t<Real, 3, QUINTIC>(c); break;
        case 4: vh_query_t<Real, 3, WENDLAND_C2>(c); break;
        default: vh_query_t<Real, 3, CUBIC_SPLINE>(c); break;
    }
}

// The whole search on the stream: clears, build, query.
void vh_enqueue(sph_vh* c) {
    if (c->timing) cudaEventRecordWithFlags(c->ev[0], c->stream, cudaEventRecordExternal);
    cudaMemsetAsync(c->work, 0, c->work_words * 4, c->stream);
    cudaMemsetAsync(c->ctl, 0, sizeof(Control), c->stream);
    const bool f32 = c->prm.precision == SPH_PREC_FP32;
    if (c->prm.dim == 3) {
        if (f32) vh_build_t<float, 3>(c);
        else vh_build_t<double, 3>(c);
    } else {
        if (f32) vh_build_t<float, 2>(c);
        else vh_build_t<double, 2>(c);
    }
    if (c->timing) cudaEventRecordWithFlags(c->ev[1], c->stream, cudaEventRecordExternal);
    if (f32) vh_query_k<float>(c);
    else vh_query_k<double>(c);
    if (c->timing) cudaEventRecordWithFlags(c->ev[2], c->stream, cudaEventRecordExternal);
}

sph_status vh_ensure_list(sph_vh* c, int maxn) {
    if (c->nl && maxn <= c->maxn) return SPH_OK;
    vh_release(c, c->nl);
    c->nl = nullptr;
    const size_t bytes = (size_t)(c->cap > 0 ? c->cap : 1) * (size_t)maxn * 4;
    c->nl = (uint32_t*)vh_alloc(c, bytes);
    if (!c->nl) {
        c->maxn = 0;
        return vfail(c, SPH_ERR_OOM, "neighbour list of " + std::to_string(bytes) + " bytes");
    }
    c->maxn = maxn;
    vh_drop_graph(c);
    return SPH_OK;
}

// One search as a captured graph (rebuilt when the particle count or the list slots
// change), or the launches themselves where capture is unavailable.
sph_status vh_run(sph_vh* c) {
    if (!c->graph || c->graph_n != c->n || c->graph_maxn != c->maxn || c->graph_timed != c->timing) {
        vh_drop_graph(c);
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
            vh_enqueue(c);
            const cudaError_t ee = cudaStreamEndCapture(c->stream, &g);
            cudaGraphExec_t ex = nullptr;
            if (ee == cudaSuccess && g && cudaGraphInstantiate(&ex, g, 0) == cudaSuccess) {
                c->graph = ex;
                c->graph_n = c->n;
                c->graph_maxn = c->maxn;
                c->graph_timed = c->timing;
            }
            if (g) cudaGraphDestroy(g);
        }
        cudaGetLastError();
    }
    if (c->graph) {
        VCK(cudaGraphLaunch(c->graph, c->stream));
    } else {
        vh_enqueue(c);
        VCK(cudaGetLastError());
    }
    return SPH_OK;
}

}  // namespace

extern "C" {

sph_status sph_vh_create(const sph_vh_params* params, int64_t capacity, void* stream,
                         sph_alloc_fn alloc, sph_free_fn free_fn, void* alloc_user, sph_vh** out) {
    if (!params || !out) return vfail(nullptr, SPH_ERR_INVALID, "NULL argument");
    *out = nullptr;
    const sph_vh_params& p = *params;
    if (p.dim != 2 && p.dim != 3) return vfail(nullptr, SPH_ERR_INVALID, "dim must be 2 or 3");
    if (p.kernel < 0 || p.kernel > 2) return vfail(nullptr, SPH_ERR_INVALID, "unknown kernel");
    if (p.precision != SPH_PREC_FP64 && p.precision != SPH_PREC_FP32)
        return vfail(nullptr, SPH_ERR_INVALID, "unknown precision");
    if (p.leaf_size < 1 || p.leaf_size > 4096)
        return vfail(nullptr, SPH_ERR_INVALID, "leaf_size must be in 1 .. 4096");
    if (capacity < 0 || capacity > (int64_t)1 << 30)
        return vfail(nullptr, SPH_ERR_INVALID, "capacity must be in 0 .. 2^30");
    if ((alloc == nullptr) != (free_fn == nullptr))
        return vfail(nullptr, SPH_ERR_INVALID, "give both allocator callbacks or neither");
    sph_vh* c = new sph_vh();
    c->prm = p;
    c->cap = capacity;
    c->alloc = alloc;
    c->free_fn = free_fn;
    c->user = alloc_user;
    int device = 0;
    cudaGetDevice(&device);
    if (cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || c->sms < 1) {
        cudaGetLastError();
        delete c;
        return vfail(nullptr, SPH_ERR_CUDA, "no CUDA device");
    }
    if (stream) {
        c->stream = (cudaStream_t)stream;
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            delete c;
            return vfail(nullptr, SPH_ERR_CUDA, "stream creation failed");
        }
        c->own_stream = true;
    }
    const size_t N = (size_t)(capacity > 0 ? capacity : 1);
    const int B = vh_bits(p.dim);
    const size_t per_level = std::min<size_t>(N, ((size_t)(1 << p.dim) * N + p.leaf_size) / (p.leaf_size + 1));
    const size_t node_cap = 1 + (size_t)B * per_level;
    c->node_cap = (uint32_t)std::min<size_t>(node_cap, 0xffffffffu);
    // the sort's look-back words for any count up to the capacity (short tiles below
    // 131,072 keys can outnumber the long tiles of a larger capacity)
    c->work_words = std::max(sort_work_words((int)N, VH_PASSES),
                             sort_work_words((int)std::min<size_t>(N, 131072), VH_PASSES));
    c->part_blocks = c->sms * 8;
    const size_t node_bytes = p.precision == SPH_PREC_FP32 ? sizeof(VhNode<float>) : sizeof(VhNode<double>);
    struct Req { void** dst; size_t bytes; };
    Req reqs[] = {
        {(void**)&c->in[0], 8 * N}, {(void**)&c->in[1], 8 * N}, {(void**)&c->in[2], 8 * N},
        {(void**)&c->in[3], 8 * N}, {(void**)&c->in[4], 8 * N},
        {(void**)&c->keys[0], 4 * N}, {(void**)&c->keys[1], 4 * N},
        {(void**)&c->vals[0], 4 * N}, {(void**)&c->vals[1], 4 * N},
        {(void**)&c->work, 4 * c->work_words},
        {&c->rec, 32 * N}, {&c->M, 8 * N},
        {&c->nodes, node_bytes * c->node_cap},
        {(void**)&c->dev, sizeof(VhDev)}, {(void**)&c->ctl, sizeof(Control)},
        {(void**)&c->part, 6 * 8 * (size_t)c->part_blocks},
        {(void**)&c->cnt, 4 * N}, {(void**)&c->rho, 8 * N},
    };
    for (const Req& r : reqs) {
        void* q = vh_alloc(c, r.bytes);
        if (!q) {
            const std::string msg = "device allocation of " + std::to_string(r.bytes) + " bytes";
            sph_vh_destroy(c);
            return vfail(nullptr, SPH_ERR_OOM, msg);
        }
        *r.dst = q;
        c->blocks.push_back(q);
    }
    if (cudaMemsetAsync(c->in[2], 0, 8 * N, c->stream) != cudaSuccess ||
        cudaMemsetAsync(c->ctl, 0, sizeof(Control), c->stream) != cudaSuccess) {
        cudaGetLastError();
        sph_vh_destroy(c);
        return vfail(nullptr, SPH_ERR_CUDA, "initial clear failed");
    }
    *out = c;
    return SPH_OK;
}

sph_status sph_vh_set(sph_vh* c, int64_t n, const double* x, const double* y, const double* z,
                      const double* h, const double* m) {
    if (!c) return vfail(c, SPH_ERR_INVALID, "ctx is NULL");
    if (n < 0 || n > c->cap) return vfail(c, SPH_ERR_INVALID, "n outside 0 .. capacity");
    if (n > 0 && (!x || !y || !h || !m || (c->prm.dim == 3 && !z)))
        return vfail(c, SPH_ERR_INVALID, "NULL array");
    for (int64_t i = 0; i < n; ++i)
        if (!(h[i] > 0.0) || !std::isfinite(h[i]))
            return vfail(c, SPH_ERR_INVALID, "h must be positive and finite (index " + std::to_string(i) + ")");
    const double* src[5] = {x, y, c->prm.dim == 3 ? z : nullptr, h, m};
    for (int k = 0; k < 5; ++k)
        if (src[k] && n > 0) VCK(cudaMemcpyAsync(c->in[k], src[k], 8 * (size_t)n, cudaMemcpyHostToDevice, c->stream));
    VCK(cudaStreamSynchronize(c->stream));
    c->n = (int)n;
    c->have = true;
    c->searched = false;
    return SPH_OK;
}

sph_status sph_vh_search(sph_vh* c) {
    if (!c) return vfail(c, SPH_ERR_INVALID, "ctx is NULL");
    if (!c->have) return vfail(c, SPH_ERR_STATE, "no particles set");
    c->searched = false;
    c->query_runs = 0;
    if (c->n == 0) {
        c->host = VhDev{};
        c->searched = true;
        return SPH_OK;
    }
    sph_status s = vh_ensure_list(c, c->maxn > 0 ? c->maxn : 64);
    if (s != SPH_OK) return s;
    for (int attempt = 0; attempt < 2; ++attempt) {
        s = vh_run(c);
        if (s != SPH_OK) return s;
        ++c->query_runs;
        Control h{};
        VCK(cudaMemcpyAsync(&h, c->ctl, sizeof h, cudaMemcpyDeviceToHost, c->stream));
        VCK(cudaMemcpyAsync(&c->host, c->dev, sizeof(VhDev), cudaMemcpyDeviceToHost, c->stream));
        VCK(cudaStreamSynchronize(c->stream));
        if (h.status & ST_TIMEOUT) return vfail(c, SPH_ERR_TIMEOUT, "a device wait of the sort ran out");
        if (!(h.status & ST_CAPACITY)) {
            c->searched = true;
            return SPH_OK;
        }
        if ((int)c->host.max_count <= c->maxn)
            return vfail(c, SPH_ERR_CAPACITY, "tree or walk capacity exceeded");
        s = vh_ensure_list(c, ((int)c->host.max_count + 7) / 8 * 8);  // slots for the largest count
        if (s != SPH_OK) return s;
    }
    return vfail(c, SPH_ERR_CAPACITY, "neighbour counts kept growing");
}

sph_status sph_vh_neighbors(sph_vh* c, int64_t* offsets, int32_t* idx, int64_t idx_capacity,
                            int64_t* nnz) {
    if (!c || !offsets || !nnz) return vfail(c, SPH_ERR_INVALID, "NULL argument");
    if (!c->searched) return vfail(c, SPH_ERR_STATE, "no search has run");
    const int n = c->n;
    std::vector<uint32_t> cnt(n), perm(n);
    if (n > 0) {
        VCK(cudaMemcpyAsync(cnt.data(), c->cnt, 4 * (size_t)n, cudaMemcpyDeviceToHost, c->stream));
        VCK(cudaMemcpyAsync(perm.data(), c->vals[c->sorted], 4 * (size_t)n, cudaMemcpyDeviceToHost, c->stream));
        VCK(cudaStreamSynchronize(c->stream));
    }
    std::vector<int64_t> rowlen(n, 0);
    for (int k = 0; k < n; ++k) rowlen[perm[k]] = cnt[k];
    offsets[0] = 0;
    for (int i = 0; i < n; ++i) offsets[i + 1] = offsets[i] + rowlen[i];
    *nnz = offsets[n];
    if (!idx) return SPH_OK;
    if (idx_capacity < offsets[n]) return vfail(c, SPH_ERR_CAPACITY, "idx buffer smaller than nnz");
    std::vector<uint32_t> nl((size_t)n * c->maxn);
    if (n > 0 && c->maxn > 0) {
        VCK(cudaMemcpyAsync(nl.data(), c->nl, nl.size() * 4, cudaMemcpyDeviceToHost, c->stream));
        VCK(cudaStreamSynchronize(c->stream));
    }
    for (int k = 0; k < n; ++k) {
        int64_t w = offsets[perm[k]];
        for (uint32_t t = 0; t < cnt[k]; ++t) idx[w++] = (int32_t)perm[nl[(size_t)t * n + k]];
    }
    return SPH_OK;
}

sph_status sph_vh_density(sph_vh* c, double* rho) {
    if (!c || !rho) return vfail(c, SPH_ERR_INVALID, "NULL argument");
    if (!c->searched) return vfail(c, SPH_ERR_STATE, "no search has run");
    if (c->n > 0) {
        VCK(cudaMemcpyAsync(rho, c->rho, 8 * (size_t)c->n, cudaMemcpyDeviceToHost, c->stream));
        VCK(cudaStreamSynchronize(c->stream));
    }
    return SPH_OK;
}

sph_status sph_vh_stats(sph_vh* c, int64_t out[8]) {
    if (!c || !out) return vfail(c, SPH_ERR_INVALID, "NULL argument");
    if (!c->searched) return vfail(c, SPH_ERR_STATE, "no search has run");
    int64_t nodes = 0;
    int deepest = 0;
    for (int l = 0; l <= VH_LEVELS; ++l) {
        nodes += c->host.level_n[l];
        if (c->host.level_n[l]) deepest = l;
    }
    out[0] = std::min<int64_t>(nodes, c->node_cap);
    out[1] = c->host.leaves;
    out[2] = deepest;
    out[3] = (int64_t)c->host.cand;
    out[4] = (int64_t)c->host.pairs;
    out[5] = c->host.max_count;
    out[6] = c->maxn;
    out[7] = c->query_runs;
    return SPH_OK;
}

sph_status sph_vh_tree(sph_vh* c, int64_t nodes_capacity, int32_t* start, int32_t* end,
                       int32_t* child, int32_t* nchild, double* lo, double* hi, double* hmax,
                       int32_t* perm) {
    if (!c) return vfail(c, SPH_ERR_INVALID, "ctx is NULL");
    if (!c->searched) return vfail(c, SPH_ERR_STATE, "no search has run");
    int64_t st[8];
    sph_vh_stats(c, st);
    const int64_t nn = st[0];
    if (nodes_capacity < nn) return vfail(c, SPH_ERR_CAPACITY, "node buffers smaller than the tree");
    const bool f32 = c->prm.precision == SPH_PREC_FP32;
    const size_t nb = f32 ? sizeof(VhNode<float>) : sizeof(VhNode<double>);
    std::vector<unsigned char> raw((size_t)nn * nb);
    if (nn > 0) VCK(cudaMemcpyAsync(raw.data(), c->nodes, raw.size(), cudaMemcpyDeviceToHost, c->stream));
    std::vector<uint32_t> p(c->n);
    if (c->n > 0) VCK(cudaMemcpyAsync(p.data(), c->vals[c->sorted], 4 * (size_t)c->n, cudaMemcpyDeviceToHost, c->stream));
    VCK(cudaStreamSynchronize(c->stream));
    for (int64_t q = 0; q < nn; ++q) {
        double a[4], b[4];
        int4 r;
        if (f32) {
            const VhNode<float>* v = (const VhNode<float>*)raw.data() + q;
            a[0] = v->lo.x; a[1] = v->lo.y; a[2] = v->lo.z; a[3] = v->lo.w;
            b[0] = v->hi.x; b[1] = v->hi.y; b[2] = v->hi.z;
            r = v->r;
        } else {
            const VhNode<double>* v = (const VhNode<double>*)raw.data() + q;
            a[0] = v->lo.x; a[1] = v->lo.y; a[2] = v->lo.z; a[3] = v->lo.w;
            b[0] = v->hi.x; b[1] = v->hi.y; b[2] = v->hi.z;
            r = v->r;
        }
        if (start) start[q] = r.x;
        if (end) end[q] = r.y;
        if (child) child[q] = r.z;
        if (nchild) nchild[q] = r.w;
        for (int d = 0; d < 3; ++d) {
            if (lo) lo[3 * q + d] = a[d];
            if (hi) hi[3 * q + d] = b[d];
        }
        if (hmax) hmax[q] = a[3];
    }
    if (perm)
        for (int k = 0; k < c->n; ++k) perm[k] = (int32_t)p[k];
    return SPH_OK;
}

sph_status sph_vh_set_timing(sph_vh* c, int32_t enable) {
    if (!c) return vfail(c, SPH_ERR_INVALID, "ctx is NULL");
    if (enable && !c->ev[0])
        for (int k = 0; k < 3; ++k) VCK(cudaEventCreate(&c->ev[k]));
    c->timing = enable != 0;
    return SPH_OK;
}

sph_status sph_vh_phase_times(sph_vh* c, float out[2]) {
    if (!c || !out) return vfail(c, SPH_ERR_INVALID, "NULL argument");
    if (!c->searched || !c->timing || c->n == 0) return vfail(c, SPH_ERR_STATE, "no timed search has run");
    VCK(cudaEventElapsedTime(&out[0], c->ev[0], c->ev[1]));
    VCK(cudaEventElapsedTime(&out[1], c->ev[1], c->ev[2]));
    return SPH_OK;
}

const char* sph_vh_last_error(const sph_vh* c) { return c ? c->err.c_str() : g_vh_error.c_str(); }

void sph_vh_destroy(sph_vh* c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    vh_drop_graph(c);
    for (int k = 0; k < 3; ++k)
        if (c->ev[k]) cudaEventDestroy(c->ev[k]);
    vh_release(c, c->nl);
    for (void* p : c->blocks) vh_release(c, p);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
}

}  // extern "C"
