// Pair loops of one right-hand-side evaluation over the cell-sorted particles
// (Sec. 3.2 groups; per-destination loop of Sec. 3.4), as kernel templates:
//  - the density pass: summation density, Eq. (2), or the continuity rate,
//    Eq. (continuity:sph), with the position-like density advance, then the EOS; or the
//    pressure rate of the EDAC form (Sec. 2.3 scheme list, the Taylor-Green runs of
//    Sec. 4.1) with the same advance of the pressure;
//  - the momentum pass: pressure Eq. (mom:sph:press), laminar viscosity
//    Eq. (mom:sph:visc), Monaghan artificial viscosity, XSPH and the body force of
//    Eq. (mom:sph), with the corrector half-kick of Sec. 2.1 and the FP64 diagnostics.
//
// Work decomposition: the density pass gives one thread to each destination, walks the
// 3^(d-1) contiguous source runs of its stencil (a tight load-test loop) and records the
// accepted sources in an interleaved neighbour list (nl[k * n + i]: lanes of a warp read
// consecutive words); its density sum and the whole momentum pass then loop over that
// list with no predicate and little divergence. In the momentum pass a group of T lanes
// (T = 1, 2, 4 or 8, the tile shape the autotuner picks) shares one destination; each
// lane keeps compensated partial sums and a fixed shuffle tree combines them, so results
// are deterministic.
#pragma once

#include <type_traits>

#include "sph_device.cuh"
#include "sph_launch.h"
#include "step_impl.cuh"
#include "stencil.cuh"
#include "reduce_impl.cuh"
#include "pair_units.h"

namespace sph {

constexpr int PAIR_THREADS = 128;
constexpr int MOM_CHUNK = 32;  // destinations a warp takes at a time (one-lane momentum pass)

// The stencil walk clipped to the support: a row (dy, dz) whose distance from the
// destination in (y, z) reaches the support radius is skipped, and in every other row the
// x cells out of reach are dropped, so only candidates that can pass the predicate are
// examined; the order of the remaining runs (and so of the neighbour list) is that of
// for_each_run. body(jb, je, sx, sy, sz) also gets the run's minimum-image shift
// (s = +L where the run wraps below the box, -L above; valid when G.run_shift). `e` holds
// the destination's distances to the lower faces of its own cell and `c` the cell sizes;
// `reach2` is the squared support radius widened by a margin far above the FP32 rounding of
// these distances, so no cell that holds a neighbour is dropped. The run of the
// destination's own row is passed as the two runs around the destination's own index
// `self`, so no candidate test has to exclude it. Returns, in ncand, the candidates of the
// full stencil (the count the interaction metric reports).
template <class Real, int DIM, class Body>
__device__ __forceinline__ void for_each_clipped_run(const Grid& G, const PairConst<Real>& K,
                                                     const uint32_t* __restrict__ off, int cx, int cy,
                                                     int cz, const float* e, const float* c,
                                                     float reach2, uint32_t& ncand, uint32_t self,
                                                     Body body) {
    constexpr int R = Stencil<DIM>::R, RZ = Stencil<DIM>::RZ;
    const int nx = G.nc[0];
#pragma unroll 1
    for (int dz = -RZ; dz <= RZ; ++dz) {
        int z = cz + dz;
        Real sz = Real(0);
        if (DIM == 3 && (z < 0 || z >= G.nc[2])) {
            if (!G.periodic[2]) continue;
            sz = z < 0 ? K.L[2] : -K.L[2];
            z = z < 0 ? z + G.nc[2] : z - G.nc[2];
        }
        // distance to the nearest face of the layer dz cells away
        const float bz = DIM == 3 ? (dz < 0 ? e[2] + (float)(-dz - 1) * c[2]
                                            : (dz > 0 ? (c[2] - e[2]) + (float)(dz - 1) * c[2] : 0.0f))
                                  : 0.0f;
#pragma unroll 1
        for (int dy = -R; dy <= R; ++dy) {
            int y = cy + dy;
            Real sy = Real(0);
            if (y < 0 || y >= G.nc[1]) {
                if (!G.periodic[1]) continue;
                sy = y < 0 ? K.L[1] : -K.L[1];
                y = y < 0 ? y + G.nc[1] : y - G.nc[1];
            }
            const float ay = dy < 0 ? e[1] + (float)(-dy - 1) * c[1]
                                    : (dy > 0 ? (c[1] - e[1]) + (float)(dy - 1) * c[1] : 0.0f);
            const float w2 = reach2 - (ay * ay + bz * bz);  // <= 0: the row is out of reach
            // cells within reach on each side of cx
            int nl = 0, nr = 0;
            if (w2 > 0.0f) {
#pragma unroll
                for (int k = 1; k <= R; ++k) {
                    const float dl = e[0] + (float)(k - 1) * c[0], dr = (c[0] - e[0]) + (float)(k - 1) * c[0];
                    nl += dl * dl < w2 ? 1 : 0;
                    nr += dr * dr < w2 ? 1 : 0;
                }
            }
            const int rowb = nx * (y + G.nc[1] * z);
            int xa = cx - R, xb = cx + R;               // full row
            int t0 = cx - nl, t1 = cx + nr;             // clipped row
            if (G.periodic[0]) {
                if (xa < 0) {
                    ncand += off[rowb + nx] - off[rowb + nx + xa];
                    if (w2 > 0.0f && t0 < 0) body(off[rowb + nx + t0], off[rowb + nx], K.L[0], sy, sz);
                    xa = 0;
                }
                if (xb >= nx) {
                    ncand += off[rowb + xb - nx + 1] - off[rowb];
                    if (w2 > 0.0f && t1 >= nx) body(off[rowb], off[rowb + t1 - nx + 1], -K.L[0], sy, sz);
                    xb = nx - 1;
                }
            } else {
                if (xa < 0) xa = 0;
                if (xb >= nx) xb = nx - 1;
            }
            const uint32_t fb = off[rowb + xa], fe = off[rowb + xb + 1];
            ncand += fe - fb;
            if (!(w2 > 0.0f)) continue;
            t0 = max(t0, xa);
            t1 = min(t1, xb);
            if (t0 > t1) continue;
            const uint32_t jb = t0 == xa ? fb : off[rowb + t0], je = t1 == xb ? fe : off[rowb + t1 + 1];
            if (dz == 0 && dy == 0) {
                // the destination's own cell: its run without the destination itself
                body(jb, self, Real(0), sy, sz);
                body(self + 1, je, Real(0), sy, sz);
            } else {
                body(jb, je, Real(0), sy, sz);
            }
        }
    }
}

// The T lanes of one destination inside a warp.
template <int T>
struct Group {
    int t;          // lane within the group
    int shift;      // first warp lane of the group
    unsigned mask;  // warp lanes of the group
    __device__ __forceinline__ Group() {
        const int lane = threadIdx.x & 31;
        t = lane & (T - 1);
        shift = lane - t;
        mask = (T == 32) ? 0xffffffffu : (((1u << T) - 1u) << shift);
    }
    __device__ __forceinline__ unsigned ballot(bool p) const {
        const unsigned b = __ballot_sync(mask, p);
        return T == 32 ? b : ((b >> shift) & ((1u << T) - 1u));
    }
    __device__ __forceinline__ void sync() const { __syncwarp(mask); }
    template <class V>
    __device__ __forceinline__ V down(V v, int o) const { return __shfl_down_sync(mask, v, o, T); }
};

// Combines the lanes' compensated partial sums into lane 0 (fixed order).
template <class Real, int T>
__device__ __forceinline__ void group_reduce(Acc<Real>& a, const Group<T>& g) {
#pragma unroll
    for (int o = T / 2; o > 0; o >>= 1) {
        const Real s2 = g.down(a.s, o);
        const Real c2 = g.down(a.c, o);
        a.add(s2);
        a.c += c2;
    }
}

// Separation of i and j with the neighbour predicate's exact arithmetic.
template <class Real, int DIM>
__device__ __forceinline__ Real separation(const typename V4<Real>::T& pi,
                                           const typename V4<Real>::T& pj, const Grid& G,
                                           const PairConst<Real>& K, Real& dx, Real& dy, Real& dz) {
    dx = min_image(rn_sub(pi.x, pj.x), G.periodic[0], K.L[0], K.halfL[0]);
    dy = min_image(rn_sub(pi.y, pj.y), G.periodic[1], K.L[1], K.halfL[1]);
    dz = DIM == 3 ? min_image(rn_sub(pi.z, pj.z), G.periodic[2], K.L[2], K.halfL[2]) : Real(0);
    return dist2<Real, DIM>(dx, dy, dz);
}

// FP32 pair sums (not the predicate): the separation of the rounded positions corrected
// by the difference of their residuals E (reorder_one). x_i - x_j of nearby floats is
// exact, so the corrected separation carries the rounding of itself rather than that of
// the positions, which is ulp(x) / r larger where |x| is much larger than the particle
// spacing (a velocity change of 1e-4 of u per step, as on fine Taylor-Green lattices, then
// comes from pair sums that cancel to 1e-2 of their terms). FP64 mode passes no E.
template <class Real, int DIM>
__device__ __forceinline__ void add_residuals(const F4* __restrict__ E, const F4& ei, uint32_t j,
                                              Real& dx, Real& dy, Real& dz) {
    if (sizeof(Real) == 4 && E) {
        const F4 ej = E[j];
        dx += (Real)(ei.x - ej.x);
        dy += (Real)(ei.y - ej.y);
        if (DIM == 3) dz += (Real)(ei.z - ej.z);
    }
}

__device__ __forceinline__ F4 residual_of(const F4* __restrict__ E, int i) {
    return E ? E[i] : F4{0.f, 0.f, 0.f, 0.f};
}

// Separation for the pair sums over a neighbour list: with MI the minimum image on the
// periodic axes (separation above), else the plain difference, which equals it wherever
// no neighbour lies across a periodic boundary.
template <class Real, int DIM, bool MI>
__device__ __forceinline__ void pair_separation(const typename V4<Real>::T& pi,
                                                const typename V4<Real>::T& pj, const Grid& G,
                                                const PairConst<Real>& K, Real& dx, Real& dy,
                                                Real& dz) {
    if (MI) {
        separation<Real, DIM>(pi, pj, G, K, dx, dy, dz);
    } else {
        dx = rn_sub(pi.x, pj.x);
        dy = rn_sub(pi.y, pj.y);
        dz = DIM == 3 ? rn_sub(pi.z, pj.z) : Real(0);
    }
}

// Whether a neighbour of destination pi, or of another destination of the warp, can lie
// across a periodic boundary: within the support (with a margin far above the rounding of
// the test) of the box faces of some periodic axis. Elsewhere every neighbour's raw
// difference is shorter than the support, so below half the period, and the minimum image
// leaves it unchanged. Decided for the whole warp, so that its lanes take one loop.
template <class Real, int DIM>
__device__ __forceinline__ bool near_periodic_face(const typename V4<Real>::T& pi, const Grid& G,
                                                   const PairConst<Real>& K) {
    bool near = false;
    if (G.periodic[0] || G.periodic[1] || (DIM == 3 && G.periodic[2])) {
        // the support radius with a 1 % margin, far above the FP32 rounding of its root
        const double reach = (double)(1.01f * sqrtf((float)K.kh2));
        const double xs[3] = {(double)pi.x, (double)pi.y, (double)pi.z};
#pragma unroll
        for (int d = 0; d < DIM; ++d)
            near |= G.periodic[d] && (xs[d] - G.lo[d] < reach || G.hi[d] - xs[d] < reach);
    }
    return __any_sync(__activemask(), near) != 0;
}

// ------------------------------------------------------------ diagnostics
// Block partials of one evaluation, 8-byte slots: momentum pass [px, py, pz, ke] (FP64
// sums), [max |u|^2, max |a|^2] (bit patterns of non-negative doubles, whose integer
// order is their numeric order), [non-finite flag]; density pass [interacting pairs,
// candidates, wall-destination pairs] (64-bit integers). Integer maxima, flags and counts
// are exact in any order and keep the scarce FP64 pipe for the sums.
struct MomDiag {
    double px, py, pz, ke;
    unsigned long long u2b, a2b;
    unsigned bad;
};

struct DensityCounts {
    unsigned long long pairs, cand, wall;
    int overflow;
};

__device__ __forceinline__ unsigned long long u64max(unsigned long long a, unsigned long long b) {
    return a > b ? a : b;
}

// Reduction of a warp's momentum diagnostics into lane 0 (fixed order).
__device__ __forceinline__ void warp_mom_diag(MomDiag& md) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        md.px += __shfl_down_sync(0xffffffffu, md.px, o);
        md.py += __shfl_down_sync(0xffffffffu, md.py, o);
        md.pz += __shfl_down_sync(0xffffffffu, md.pz, o);
        md.ke += __shfl_down_sync(0xffffffffu, md.ke, o);
        md.u2b = u64max(md.u2b, __shfl_down_sync(0xffffffffu, md.u2b, o));
        md.a2b = u64max(md.a2b, __shfl_down_sync(0xffffffffu, md.a2b, o));
        md.bad |= __shfl_down_sync(0xffffffffu, md.bad, o);
    }
}

// Block reduction of the momentum diagnostics held by the first NW warps (fixed order);
// thread 0 writes the 7 slots to out.
template <int NW>
__device__ __forceinline__ void block_mom_diag(MomDiag md, double* out, MomDiag* red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (warp < NW) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            md.px += __shfl_down_sync(0xffffffffu, md.px, o);
            md.py += __shfl_down_sync(0xffffffffu, md.py, o);
            md.pz += __shfl_down_sync(0xffffffffu, md.pz, o);
            md.ke += __shfl_down_sync(0xffffffffu, md.ke, o);
            md.u2b = u64max(md.u2b, __shfl_down_sync(0xffffffffu, md.u2b, o));
            md.a2b = u64max(md.a2b, __shfl_down_sync(0xffffffffu, md.a2b, o));
            md.bad |= __shfl_down_sync(0xffffffffu, md.bad, o);
        }
        if (lane == 0) red[warp] = md;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        MomDiag t = red[0];
        for (int w = 1; w < NW; ++w) {
            t.px += red[w].px;
            t.py += red[w].py;
            t.pz += red[w].pz;
            t.ke += red[w].ke;
            t.u2b = u64max(t.u2b, red[w].u2b);
            t.a2b = u64max(t.a2b, red[w].a2b);
            t.bad |= red[w].bad;
        }
        out[0] = t.px;
        out[1] = t.py;
        out[2] = t.pz;
        out[3] = t.ke;
        out[4] = __longlong_as_double((long long)t.u2b);
        out[5] = __longlong_as_double((long long)t.a2b);
        out[6] = __longlong_as_double((long long)t.bad);
    }
    __syncthreads();
}

// Block sums of the density-pass counters (NTH threads); thread 0 writes 3 slots to out.
template <int NTH>
__device__ __forceinline__ void block_counts(const DensityCounts& dc, double* out,
                                             unsigned long long (*red)[3]) {
    unsigned long long v[3] = {dc.pairs, dc.cand, dc.wall};
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int k = 0; k < 3; ++k) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < 3; ++k) red[warp][k] = v[k];
    __syncthreads();
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            unsigned long long t = red[0][k];
            for (int w = 1; w < NTH / 32; ++w) t += red[w][k];
            out[k] = __longlong_as_double((long long)t);
        }
    __syncthreads();
}

// Reduction of the block partials of both passes (NTH threads, fixed order) into
// out[10] = px py pz ke max|u|^2 max|a|^2 bad pairs candidates wall-pairs (thread 0).
template <int NTH>
__device__ __forceinline__ void reduce_partials(const double* pm, int pm_stride, int nbm,
                                                const double* pd, int pd_stride, int nbd,
                                                double* out, MomDiag* red,
                                                unsigned long long (*cred)[3]) {
    MomDiag md{0, 0, 0, 0, 0ull, 0ull, 0u};
    for (int b = threadIdx.x; b < nbm; b += NTH) {
        const volatile double* p = pm + (size_t)b * pm_stride;
        md.px += p[0];
        md.py += p[1];
        md.pz += p[2];
        md.ke += p[3];
        md.u2b = u64max(md.u2b, (unsigned long long)__double_as_longlong(p[4]));
        md.a2b = u64max(md.a2b, (unsigned long long)__double_as_longlong(p[5]));
        md.bad |= (unsigned)__double_as_longlong(p[6]);
    }
    DensityCounts dc{0ull, 0ull, 0ull, 0};
    for (int b = threadIdx.x; b < nbd; b += NTH) {
        const volatile double* p = pd + (size_t)b * pd_stride;
        dc.pairs += (unsigned long long)__double_as_longlong(p[0]);
        dc.cand += (unsigned long long)__double_as_longlong(p[1]);
        dc.wall += (unsigned long long)__double_as_longlong(p[2]);
    }
    double m[7], c[3];
    block_mom_diag<NTH / 32>(md, m, red);
    block_counts<NTH>(dc, c, cred);
    if (threadIdx.x == 0) {
        for (int k = 0; k < 4; ++k) out[k] = m[k];
        out[4] = __longlong_as_double(__double_as_longlong(m[4]));
        out[5] = __longlong_as_double(__double_as_longlong(m[5]));
        out[6] = (double)(unsigned)__double_as_longlong(m[6]);
        for (int k = 0; k < 3; ++k) out[7 + k] = (double)(unsigned long long)__double_as_longlong(c[k]);
    }
}

// ---------------------------------------------------------------- density pass
// A group of T lanes per destination (T = 1, 2, 4 or 8). (1) Neighbour scan: the 3^(d-1)
// contiguous source runs of the destination's stencil, T candidates at a time (lane t
// takes the t-th), the exact neighbour predicate, and the accepted sources appended to
// the interleaved neighbour list nl[k * n + i] (k < maxn; cnt[i] entries) in candidate
// order: a ballot over the group gives each accepted lane its slot, so the list is the
// same for every T. Continuity mode lists interacting sources only (a wall destination
// takes fluid sources); summation mode lists every neighbour. (2) The density group
// over the list, lane t taking every T-th entry with compensated partial sums combined
// by a fixed shuffle tree:
//  summation (Eq. 2): rho_i = sum_j m_j W_ij, self term included;
//  continuity (Eq. continuity:sph): arho_i = sum_j m_j v_ij . grad_i W_ij and, inside a
//    step, rho_i += dt arho_i (density advanced like the positions, Sec. 2.1 reading).
// (3) The epilogue (FP64 density update, the Tait EOS of Eq. eos for the shadow
// p / rho^2, in the pair-loop precision): with T > 1 the destinations of a block tile
// hand their sums through shared memory to one thread each, so the FP64 work runs on
// full warps. Counts interacting pairs (not both walls), candidates and the interacting
// pairs with a wall destination. A list overflow raises ST_CAPACITY (the evaluation is
// then invalid and the step reports it).
template <int T>
__device__ __forceinline__ uint32_t group_sum_u32(uint32_t v, const Group<T>& g) {
#pragma unroll
    for (int o = T / 2; o > 0; o >>= 1) v += g.down(v, o);
    return v;
}

// Step (2) for destination i over its k list entries (lane t of the group takes every
// T-th entry); the compensated sum is valid in lane t after the loop, before the group
// reduction.
template <class Real, int DIM, int KERNEL, int T>
__device__ __forceinline__ void density_list_sum(int i, const Group<T>& g,
                                                 const typename V4<Real>::T& pi,
                                                 const typename V4<Real>::T* __restrict__ P,
                                                 const typename V4<Real>::T* __restrict__ Q,
                                                 const F4* __restrict__ E, int n, const Grid& G,
                                                 const PairConst<Real>& K,
                                                 const uint32_t* __restrict__ nl, uint32_t k,
                                                 Acc<Real>& sum) {
    using yes = std::true_type;
    using no = std::false_type;
    const bool edac = (K.flags & F_EDAC) != 0;
    const bool summation = !(K.flags & (F_CONTINUITY | F_EDAC));
    sum.zero();
    const typename V4<Real>::T qi = Q[i];
    const F4 ei = residual_of(E, i);
    // the next list entry is fetched one iteration ahead, so its load overlaps this
    // iteration's source loads and arithmetic
    // the loop without the minimum image unless a neighbour can lie across a periodic
    // boundary (the same values: the image is the identity there)
    auto sum_loop = [&](auto mi_tag) {
    constexpr bool MI = decltype(mi_tag)::value;
    uint32_t j_next = g.t < k ? nl[(size_t)g.t * n + i] : 0u;
#pragma unroll 2
    for (uint32_t kk = g.t; kk < k; kk += T) {
        const uint32_t j = j_next;
        if (kk + T < k) j_next = nl[(size_t)(kk + T) * n + i];
        const typename V4<Real>::T pj = P[j];
        Real dx, dy, dz;
        pair_separation<Real, DIM, MI>(pi, pj, G, K, dx, dy, dz);
        add_residuals<Real, DIM>(E, ei, j, dx, dy, dz);
        const Real r2 = dist2<Real, DIM>(dx, dy, dz);
        const Real q = PairMath<Real>::sqrt(r2) * K.inv_h;
        if (summation) {
            sum.add(fabs(pj.w) * K.wfac * kernel_w<Real, KERNEL>(q));
        } else {
            const typename V4<Real>::T qj = Q[j];
            const Real Gk = K.gfac * kernel_f<Real, KERNEL>(q);
            const Real vdotr = dot_rn<Real, DIM>(qi.x - qj.x, qi.y - qj.y, qi.z - qj.z, dx, dy, dz);
            if (edac)  // Q.w holds the pressure p^n: c0^2 u_ij . grad W + (2 nu_e / rho0) p_ij r . grad W / (r^2 + 0.01 h^2)
                sum.add(fabs(pj.w) * Gk *
                        fma_rn(K.c02, vdotr, K.edac_d * (qi.w - qj.w) * r2 * PairMath<Real>::rcp(r2 + K.av_h2)));
            else
                sum.add(fabs(pj.w) * Gk * vdotr);
        }
    }
    };
    if (near_periodic_face<Real, DIM>(pi, G, K)) sum_loop(yes());
    else sum_loop(no());
}

// Steps (1) and (2) for destination i; the compensated sum is valid in lane 0.
template <class Real, int DIM, int KERNEL, int T>
__device__ __forceinline__ void density_scan_sum(int i, const Group<T>& g, uint32_t key,
                                                 const typename V4<Real>::T* __restrict__ P,
                                                 const typename V4<Real>::T* __restrict__ Q,
                                                 const F4* __restrict__ E,
                                                 const uint32_t* __restrict__ off, int n,
                                                 const Grid& G, const PairConst<Real>& K,
                                                 uint32_t* __restrict__ nl,
                                                 uint32_t* __restrict__ cnt, int maxn,
                                                 DensityCounts& dc, uint32_t* pcount_i,
                                                 Acc<Real>& sum) {
    const bool edac = (K.flags & F_EDAC) != 0;
    const bool summation = !(K.flags & (F_CONTINUITY | F_EDAC));
    const typename V4<Real>::T pi = P[i];
    const bool fluid_i = pi.w > Real(0);
    int cx, cy, cz;
    cell_of_key(G, key, cx, cy, cz);
    uint32_t k = 0, npairs = 0, ncand = 0;
    const unsigned below = (1u << g.t) - 1u;
    // candidates of one run: SHIFT adds the run's minimum-image shift (exact: adding 0
    // changes nothing but the sign of a zero), MINIMG applies the per-pair minimum image,
    // SELF tests j != i (the clipped walk leaves i out of its runs instead); MODE 0 lists
    // every neighbour and counts the interacting ones (summation density), 1 lists
    // neighbours of a warp of fluid destinations (all interact), 2 lists the interacting
    // neighbours (a wall destination takes fluid sources only). In modes 1 and 2 every
    // listed pair interacts, so the interaction count is the list count.
    auto scan = [&](uint32_t jb, uint32_t je, Real sx, Real sy, Real sz, auto shift_tag,
                    auto minimg_tag, auto self_tag, auto mode_tag) {
        constexpr bool SHIFT = decltype(shift_tag)::value;
        constexpr bool MINIMG = decltype(minimg_tag)::value;
        constexpr bool SELF = decltype(self_tag)::value;
        constexpr int MODE = decltype(mode_tag)::value;
#pragma unroll 2
        for (uint32_t c = jb; c < je; c += T) {
            const uint32_t j = c + g.t;
            // written as predicates: the loop body is a straight line (no per-candidate
            // branches but the loop's own)
            bool listed = false, inter = false;
            if (T == 1 || j < je) {
                const typename V4<Real>::T pj = P[j];
                Real dx = rn_sub(pi.x, pj.x), dy = rn_sub(pi.y, pj.y);
                Real dz = DIM == 3 ? rn_sub(pi.z, pj.z) : Real(0);
                if (MINIMG) {
                    dx = min_image(dx, G.periodic[0], K.L[0], K.halfL[0]);
                    dy = min_image(dy, G.periodic[1], K.L[1], K.halfL[1]);
                    if (DIM == 3) dz = min_image(dz, G.periodic[2], K.L[2], K.halfL[2]);
                }
                if (SHIFT) {
                    dx = rn_add(dx, sx);
                    dy = rn_add(dy, sy);
                    if (DIM == 3) dz = rn_add(dz, sz);
                }
                const Real r2 = dist2<Real, DIM>(dx, dy, dz);
                const bool hit = SELF ? ((r2 < K.kh2) & ((int)j != i)) : (r2 < K.kh2);
                if (MODE == 0) {
                    listed = hit;
                    inter = hit & (fluid_i | (pj.w > Real(0)));
                } else if (MODE == 1) {
                    listed = hit;
                } else {
                    listed = hit & (fluid_i | (pj.w > Real(0)));
                }
            }
            if (MODE == 0) npairs += inter ? 1u : 0u;
            if (T == 1) {
                if (listed & (k < (uint32_t)maxn)) nl[(size_t)k * n + i] = j;
                k += listed ? 1u : 0u;
            } else {
                const unsigned m = g.ballot(listed);
                const uint32_t pos = k + __popc(m & below);
                if (listed & (pos < (uint32_t)maxn)) nl[(size_t)pos * n + i] = j;
                k += __popc(m);
            }
        }
    };
    using yes = std::true_type;
    using no = std::false_type;
    using M0 = std::integral_constant<int, 0>;
    using M1 = std::integral_constant<int, 1>;
    using M2 = std::integral_constant<int, 2>;
    const bool all_fluid = __all_sync(__activemask(), fluid_i) != 0;
    const int mode = summation ? 0 : (all_fluid ? 1 : 2);
    // mode 1 only on the common path (unshifted runs of the clipped walk): elsewhere mode 2
    // lists the same pairs
    auto scan_mode = [&](uint32_t jb, uint32_t je, Real sx, Real sy, Real sz, auto shift_tag,
                         auto minimg_tag, auto self_tag) {
        constexpr bool COMMON = !decltype(shift_tag)::value && !decltype(minimg_tag)::value;
        if (mode == 0) scan(jb, je, sx, sy, sz, shift_tag, minimg_tag, self_tag, M0());
        else if (COMMON && mode == 1) scan(jb, je, sx, sy, sz, shift_tag, minimg_tag, self_tag, M1());
        else scan(jb, je, sx, sy, sz, shift_tag, minimg_tag, self_tag, M2());
    };
    uint32_t nfull = 0;  // candidates of the full stencil, self included
    if (G.run_shift) {
        // distances to the lower faces of the own cell (FP64, then FP32 with a margin)
        float e[3] = {0.f, 0.f, 0.f}, cs[3] = {1.f, 1.f, 1.f};
        const int cc[3] = {cx, cy, cz};
        const double xs[3] = {(double)pi.x, (double)pi.y, (double)pi.z};
        for (int d = 0; d < DIM; ++d) {
            e[d] = (float)((xs[d] - G.lo[d]) - (double)cc[d] * G.cs[d]);
            cs[d] = (float)G.cs[d];
        }
        const float reach2 = (float)K.kh2 * 1.002f;
        for_each_clipped_run<Real, DIM>(G, K, off, cx, cy, cz, e, cs, reach2, nfull, (uint32_t)i,
                                        [&](uint32_t jb, uint32_t je, Real sx, Real sy, Real sz) {
            if (sx == Real(0) && sy == Real(0) && sz == Real(0)) scan_mode(jb, je, sx, sy, sz, no(), no(), no());
            else scan_mode(jb, je, sx, sy, sz, yes(), no(), no());
        });
    } else {
        for_each_run<DIM>(G, off, cx, cy, cz, [&](uint32_t jb, uint32_t je) {
            nfull += je - jb;
            scan_mode(jb, je, Real(0), Real(0), Real(0), no(), yes(), yes());
        });
    }
    if (mode != 0) npairs = g.t == 0 ? k : 0u;  // every listed pair interacts
    if (g.t == 0) ncand = nfull - 1u;  // the destination itself is in its own cell
    if (k > (uint32_t)maxn) {
        dc.overflow = 1;
        k = maxn;
    }
    if (g.t == 0) cnt[i] = k;
    g.sync();  // the list entries of the other lanes are visible from here on
    density_list_sum<Real, DIM, KERNEL, T>(i, g, pi, P, Q, E, n, G, K, nl, k, sum);
    if (T > 1) group_reduce<Real, T>(sum, g);
    dc.pairs += npairs;
    dc.cand += ncand;
    if (!fluid_i) dc.wall += npairs;
    if (pcount_i) {
        const uint32_t np = group_sum_u32<T>(npairs, g), nc = group_sum_u32<T>(ncand, g);
        if (g.t == 0) {
            pcount_i[0] = np;
            pcount_i[1] = nc;
        }
    }
}

// Step (3) for destination i with the density-group value `value` (one thread).
template <class Real, int KERNEL>
__device__ __forceinline__ void density_finish(int i, double value, Real mi,
                                               typename V4<Real>::T* __restrict__ Q,
                                               Real* __restrict__ R, const PairConst<Real>& K,
                                               const StepConst& C, const ParticleSet& S,
                                               double dt, int kick) {
    if (K.flags & F_EDAC) {
        // the EDAC pressure advanced like the continuity density; the density stays rho0,
        // and Q.w keeps p^n, which the other destinations of this pass read
        double p = S.p[i];
        if (kick) p = fma_rn(dt, value, p);
        S.p[i] = p;
        S.arho[i] = value;
        R[i] = (Real)(p * C.inv_rho0 * C.inv_rho0);
        return;
    }
    double rho, arho;
    if (!(K.flags & F_CONTINUITY)) {
        rho = value + (double)(fabs(mi) * K.wfac * kernel_w<Real, KERNEL>(Real(0)));
        arho = 0.0;
    } else {
        arho = value;
        rho = S.rho[i];
        if (kick) rho = fma_rn(dt, arho, rho);
    }
    S.rho[i] = rho;
    S.arho[i] = arho;
    reinterpret_cast<Real*>(&Q[i])[3] = (Real)rho;
    R[i] = pressure_over_rho2<Real>(rho, C);
}

// Hand-off of the compensated sums of a block tile to the epilogue threads (T > 1; a
// single placeholder entry when T = 1).
template <class Real, int GD>
struct DensitySmem {
    Real s[GD], c[GD];
};

// Density pass over destinations [tile * GD, (tile + 1) * GD) for tile = block,
// block + nblocks, ... (GD = NTH / T); each destination finds its instance's constants in
// the table (one entry for a single problem). pcount (batches): per-particle counts.
template <class Real, int DIM, int KERNEL, int T, int NTH, bool SINGLE = false>
__device__ __forceinline__ void density_tiles(int block, int nblocks,
                                              const typename V4<Real>::T* __restrict__ P,
                                              typename V4<Real>::T* __restrict__ Q,
                                              Real* __restrict__ R, const F4* __restrict__ E,
                                              const uint32_t* __restrict__ skeys,
                                              const uint32_t* __restrict__ off, int n,
                                              const Inst<Real>* __restrict__ tab,
                                              const uint32_t* __restrict__ cell_bounds, int ninst,
                                              const double* __restrict__ idt, const ParticleSet& S,
                                              int kick, uint32_t* __restrict__ nl,
                                              uint32_t* __restrict__ cnt, int maxn,
                                              uint32_t* __restrict__ pcount, DensityCounts& dc,
                                              DensitySmem<Real, T == 1 ? 1 : NTH / T>& sm,
                                              const Inst<Real>* I0 = nullptr,
                                              unsigned int* next = nullptr) {
    constexpr int GD = NTH / T;
    const Group<T> g;
    const int grp = threadIdx.x / T;
    if (T == 1 && next) {
        // each warp takes the next chunk of 32 destinations from a counter (single problems:
        // chunks differ in cost, most of all where wall destinations list fluid sources only;
        // the counts this pass accumulates are integers, so their sum does not depend on the
        // assignment)
        const int lane = threadIdx.x & 31;
        for (;;) {
            unsigned int c = 0u;
            if (lane == 0) c = atomicAdd(next, 1u);
            c = __shfl_sync(0xffffffffu, c, 0);
            if ((long long)c * 32 >= n) break;
            const int i = (int)c * 32 + lane;
            if (i < n) {
                const uint32_t key = skeys[i];
                const int inst = SINGLE ? 0 : find_instance(cell_bounds, ninst, key);
                const Inst<Real>& I = SINGLE ? *I0 : tab[inst];
                Acc<Real> sum;
                density_scan_sum<Real, DIM, KERNEL, T>(i, g, key - I.cell_base, P, Q, E, off + I.cell_base,
                                                       n, I.G, I.K, nl, cnt, maxn, dc,
                                                       pcount ? pcount + 2 * (size_t)i : nullptr, sum);
                density_finish<Real, KERNEL>(i, sum.value(), P[i].w, Q, R, I.K, I.C, S, idt[inst], kick);
            }
        }
        return;
    }
    for (int tile = block; (long long)tile * GD < n; tile += nblocks) {
        const int i = tile * GD + grp;
        if (i < n) {
            const uint32_t key = skeys[i];
            const int inst = SINGLE ? 0 : find_instance(cell_bounds, ninst, key);
            const Inst<Real>& I = SINGLE ? *I0 : tab[inst];
            Acc<Real> sum;
            density_scan_sum<Real, DIM, KERNEL, T>(i, g, key - I.cell_base, P, Q, E, off + I.cell_base,
                                                   n, I.G, I.K, nl, cnt, maxn, dc,
                                                   pcount ? pcount + 2 * (size_t)i : nullptr, sum);
            if (T == 1) {
                density_finish<Real, KERNEL>(i, sum.value(), P[i].w, Q, R, I.K, I.C, S, idt[inst], kick);
            } else if (g.t == 0) {
                sm.s[grp] = sum.s;
                sm.c[grp] = sum.c;
            }
        }
        if (T > 1) {
            __syncthreads();
            const int e = tile * GD + threadIdx.x;
            if (threadIdx.x < GD && e < n) {
                const int inst = SINGLE ? 0 : find_instance(cell_bounds, ninst, skeys[e]);
                const Inst<Real>& I = SINGLE ? *I0 : tab[inst];
                Acc<Real> a;
                a.s = sm.s[threadIdx.x];
                a.c = sm.c[threadIdx.x];
                density_finish<Real, KERNEL>(e, a.value(), P[e].w, Q, R, I.K, I.C, S, idt[inst], kick);
            }
            __syncthreads();
        }
    }
}

// Density pass kernel. Single problems write block counts to pd; batches per-particle
// counts to pcount for the per-instance reduction.
// SINGLE: a single problem, whose constants come by value in the parameter bank (I0), so
// that the pair arithmetic reads them as constant operands instead of holding them in
// registers; batches read their instance's entry of the table. The single-problem FP32 form
// is bounded to 8 or 9 blocks of 128 per SM (density_single_blocks), which it fits without
// spills.
template <int DIM, int KERNEL, int T>
constexpr int density_single_blocks() {
    // 9 blocks (56 registers) for the one-lane 3D passes of the Wendland C2 and cubic spline
    // kernels: 3 % faster than 8 on the 3D dam break and the falling cube, although at 56
    // registers the compiler recomputes FP64 values of the scan loop that 60 let it hold.
    // 8 blocks (60 registers) elsewhere: at 9 the quintic's 3D pass (Taylor-Green 3D) ran
    // 3.4 % slower and a 2D pass (the dam break at 4 lanes) 1 % slower.
    return DIM == 3 && T == 1 && KERNEL != QUINTIC ? 9 : 8;
}

template <class Real, int DIM, int KERNEL, int T, bool SINGLE>
__global__ void __launch_bounds__(PAIR_THREADS,
                                  sizeof(Real) == 4 ? (SINGLE ? density_single_blocks<DIM, KERNEL, T>() : 7) : 6)
k_density(const __grid_constant__ Inst<Real> I0,
          const typename V4<Real>::T* __restrict__ P, typename V4<Real>::T* __restrict__ Q,
          Real* __restrict__ R, const F4* __restrict__ E, const uint32_t* __restrict__ skeys,
          const uint32_t* __restrict__ off,
          int n, const Inst<Real>* __restrict__ tab, const uint32_t* __restrict__ cell_bounds,
          int ninst, const double* __restrict__ idt, ParticleSet S, Control* ctl, int kick,
          uint32_t* __restrict__ nl, uint32_t* __restrict__ cnt, int maxn,
          double* __restrict__ pd, uint32_t* __restrict__ pcount, int dyn) {
    __shared__ DensitySmem<Real, T == 1 ? 1 : PAIR_THREADS / T> sm;
    __shared__ unsigned long long cred[PAIR_THREADS / 32][3];
    // a block that starts after an earlier one raised a status (a list overflow) does no
    // work, but still counts itself done below, so the chunk counter is reset all the same
    const bool skip = ctl->status != 0u;
    DensityCounts dc{0ull, 0ull, 0ull, 0};
    if (!skip)
        density_tiles<Real, DIM, KERNEL, T, PAIR_THREADS, SINGLE>(blockIdx.x, gridDim.x, P, Q, R, E, skeys,
                                                                  off, n, tab, cell_bounds, ninst, idt, S, kick,
                                                                  nl, cnt, maxn, pcount, dc, sm, &I0,
                                                                  T == 1 && (dyn & 1) ? &ctl->dens_next
                                                                                      : nullptr);
    if (T == 1 && (dyn & 1)) {  // the last block done resets the chunk counter for the next launch
        __syncthreads();
        if (threadIdx.x == 0) {
            const unsigned int d = atomicAdd(&ctl->dens_done, 1u);
            if (d == gridDim.x - 1) {
                ctl->dens_next = 0u;
                ctl->dens_done = 0u;
            }
        }
    }
    if (skip) return;
    if (dc.overflow) atomicOr(&ctl->status, ST_CAPACITY);
    if (pd) block_counts<PAIR_THREADS>(dc, pd + (size_t)blockIdx.x * 4, cred);
}

// ------------------------------------------------------------- momentum pass
// Fluid destinations only (walls are static), over the neighbour list of the density
// pass: T lanes per destination take every T-th list entry (the tile shape the autotuner
// picks) and combine their compensated partial sums with a fixed shuffle tree. The
// epilogue (FP64 rates, the corrector half-kick u^{n+1} = u^{n+1/2} + dt/2 a^{n+1} inside
// a step, the FP64 diagnostics) runs on one thread per destination: with T > 1 the sums
// pass through shared memory so the FP64 work runs on full warps. With finalize (single
// problems) the last block to finish reduces the block partials of both passes in a fixed
// order (deterministic) and writes the record, history entry, next dt and status.

// Pair sums of destination i (fluid) into acc[0..5] = a_x a_y a_z xsph_x xsph_y xsph_z,
// valid in lane 0.
template <class Real, int DIM, int KERNEL, int T>
__device__ __forceinline__ void momentum_sums(int i, const Group<T>& g,
                                              const typename V4<Real>::T& pi,
                                              const typename V4<Real>::T* __restrict__ P,
                                              const typename V4<Real>::T* __restrict__ Q,
                                              const Real* __restrict__ R,
                                              const F4* __restrict__ E, int n, const Grid& G,
                                              const PairConst<Real>& K,
                                              const uint32_t* __restrict__ nl,
                                              const uint32_t* __restrict__ cnt, Acc<Real>* acc) {
    const int flags = K.flags;
    const typename V4<Real>::T qi = Q[i];
    const F4 ei = residual_of(E, i);
    const Real pri = R[i];
#pragma unroll
    for (int k = 0; k < 6; ++k) acc[k].zero();
    const uint32_t ni = cnt[i];
    // without the minimum image unless a neighbour can lie across a periodic boundary
    auto pair_loop = [&](auto mi_tag) {
    constexpr bool MI = decltype(mi_tag)::value;
    // the list's last reader: its entries are fetched one entry ahead and marked for early
    // eviction (streaming loads), leaving the caches to the source records
    uint32_t j_next = g.t < ni ? __ldcs(&nl[(size_t)g.t * n + i]) : 0u;
    for (uint32_t kk = g.t; kk < ni; kk += T) {
        const uint32_t j = j_next;
        if (kk + T < ni) j_next = __ldcs(&nl[(size_t)(kk + T) * n + i]);
        const typename V4<Real>::T pj = P[j];
        Real dx, dy, dz;
        pair_separation<Real, DIM, MI>(pi, pj, G, K, dx, dy, dz);
        add_residuals<Real, DIM>(E, ei, j, dx, dy, dz);
        const Real r2 = dist2<Real, DIM>(dx, dy, dz);
        const typename V4<Real>::T qj = Q[j];
        const Real mj = fabs(pj.w);
        const Real q = PairMath<Real>::sqrt(r2) * K.inv_h;
        const Real Gk = K.gfac * kernel_f<Real, KERNEL>(q);  // grad_i W = Gk (x_i - x_j)
        const Real vx = qi.x - qj.x, vy = qi.y - qj.y, vz = DIM == 3 ? qi.z - qj.z : Real(0);
        Real coef = pri + R[j];
        // EDAC: the density is rho0 (Q.w holds the pressure)
        const Real inv_rhobar = (flags & F_EDAC) ? K.inv_rho0 : PairMath<Real>::rcp(Real(0.5) * (qi.w + qj.w));
        if (flags & F_AV) {
            const Real vdotr = dot_rn<Real, DIM>(vx, vy, vz, dx, dy, dz);
            if (vdotr < Real(0)) {
                const Real mu = K.h * vdotr * PairMath<Real>::rcp(r2 + K.av_h2);
                coef -= K.alpha_c0 * mu * inv_rhobar;
            }
        }
        const Real cg = -mj * coef * Gk;
        Real cv = Real(0);
        // 4 nu m_j / (rho_i + rho_j) = 2 nu m_j / rhobar
        if (flags & F_LAMINAR)
            cv = mj * (Real(0.5) * K.nu4) * inv_rhobar * Gk * r2 * PairMath<Real>::rcp(r2 + K.eta_h2);
        acc[0].add(fma_rn(cg, dx, cv * vx));
        acc[1].add(fma_rn(cg, dy, cv * vy));
        if (DIM == 3) acc[2].add(fma_rn(cg, dz, cv * vz));
        if ((flags & F_XSPH) && pj.w > Real(0)) {
            const Real fx = K.xsph * mj * inv_rhobar * (K.wfac * kernel_w<Real, KERNEL>(q));
            acc[3].add(-fx * vx);
            acc[4].add(-fx * vy);
            if (DIM == 3) acc[5].add(-fx * vz);
        }
    }
    };
    if (near_periodic_face<Real, DIM>(pi, G, K)) pair_loop(std::true_type());
    else pair_loop(std::false_type());
    if (T > 1) {
        group_reduce<Real, T>(acc[0], g);
        group_reduce<Real, T>(acc[1], g);
        if (DIM == 3) group_reduce<Real, T>(acc[2], g);
        if (flags & F_XSPH) {
            group_reduce<Real, T>(acc[3], g);
            group_reduce<Real, T>(acc[4], g);
            if (DIM == 3) group_reduce<Real, T>(acc[5], g);
        }
    }
}

// Epilogue of destination i (one thread): FP64 rates + body force, corrector half-kick,
// diagnostics. Walls: rates zero, static.
template <int DIM>
__device__ __forceinline__ void momentum_finish(int i, bool fluid, const double* a_in,
                                                const double* xs_in, const StepConst& C,
                                                const ParticleSet& S, double dt, int kick,
                                                MomDiag& md) {
    // every load before any store: the state arrays could alias as far as the compiler
    // knows, and interleaving would serialise the round trips of the epilogue
    const double rho = S.rho[i];
    if (!fluid) {
        for (int d = 0; d < DIM; ++d) {
            S.a[d][i] = 0.0;
            S.xs[d][i] = 0.0;
        }
        if (!isfinite(rho)) md.bad = 1u;
        return;
    }
    double u[3] = {0, 0, 0}, x[3] = {0, 0, 0};
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
        u[d] = S.u[d][i];
        x[d] = S.x[d][i];
    }
    const double m = S.m[i];
    double u2 = 0, a2 = 0;
    bool bad = false;
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
        const double a = a_in[d] + C.g[d];
        S.a[d][i] = a;
        S.xs[d][i] = xs_in[d];
        if (kick) {
            u[d] = fma_rn(0.5 * dt, a, u[d]);
            S.u[d][i] = u[d];
        }
        u2 = fma_rn(u[d], u[d], u2);
        a2 = fma_rn(a, a, a2);
        bad |= !isfinite(u[d]) || !isfinite(x[d]);
    }
    bad |= !isfinite(rho) || !isfinite(a2);
    md.px = fma_rn(m, u[0], md.px);
    md.py = fma_rn(m, u[1], md.py);
    md.pz = fma_rn(m, u[2], md.pz);
    md.ke = fma_rn(0.5 * m, u2, md.ke);
    if (bad) md.bad = 1u;
    else {
        md.u2b = u64max(md.u2b, (unsigned long long)__double_as_longlong(u2));
        md.a2b = u64max(md.a2b, (unsigned long long)__double_as_longlong(a2));
    }
}

// Hand-off of the 6 compensated sums (s, c) of a block tile to the epilogue threads
// (T > 1; a single placeholder entry when T = 1).
template <class Real, int GM>
struct MomSmem {
    Real v[12][GM];
    unsigned char fluid[GM];
};

// Momentum pass over destinations [tile * GM, (tile + 1) * GM) for tile = block,
// block + nblocks, ... (GM = NTH / T).
template <class Real, int DIM, int KERNEL, int T, int NTH, bool SINGLE = false>
__device__ __forceinline__ void momentum_tiles(int block, int nblocks,
                                               const typename V4<Real>::T* __restrict__ P,
                                               const typename V4<Real>::T* __restrict__ Q,
                                               const Real* __restrict__ R, const F4* __restrict__ E,
                                               const uint32_t* __restrict__ skeys, int n,
                                               const Inst<Real>* __restrict__ tab,
                                               const uint32_t* __restrict__ cell_bounds, int ninst,
                                               const double* __restrict__ idt, const ParticleSet& S,
                                               int kick, const uint32_t* __restrict__ nl,
                                               const uint32_t* __restrict__ cnt, MomDiag& md,
                                               MomSmem<Real, T == 1 ? 1 : NTH / T>& sm,
                                               const Inst<Real>* I0 = nullptr,
                                               unsigned int* next = nullptr,
                                               double* __restrict__ cpart = nullptr) {
    constexpr int GM = NTH / T;
    const Group<T> g;
    const int grp = threadIdx.x / T;
    if (T == 1 && next) {
        // each warp takes the next chunk of MOM_CHUNK destinations (MOM_CHUNK / 32 rows of the
        // warp) from a counter: chunks of wall destinations (no pair sums) and of fluid ones
        // differ widely in cost. The diagnostics of a chunk are reduced over its lanes in a
        // fixed order and written to the chunk's slot of cpart (when given), so that their sum
        // does not depend on which warp took which chunk.
        const int lane = threadIdx.x & 31;
        for (;;) {
            unsigned int c = 0u;
            if (lane == 0) c = atomicAdd(next, 1u);
            c = __shfl_sync(0xffffffffu, c, 0);
            if ((long long)c * MOM_CHUNK >= n) break;
            MomDiag mc{0, 0, 0, 0, 0ull, 0ull, 0u};
#pragma unroll 1
            for (int r = 0; r < MOM_CHUNK / 32; ++r) {
                const long long il = (long long)c * MOM_CHUNK + r * 32 + lane;
                if (il >= n) break;
                const int i = (int)il;
                const int inst = SINGLE ? 0 : find_instance(cell_bounds, ninst, skeys[i]);
                const Inst<Real>& I = SINGLE ? *I0 : tab[inst];
                const typename V4<Real>::T pi = P[i];
                const bool fluid = pi.w > Real(0);
                Acc<Real> acc[6];
                if (fluid) momentum_sums<Real, DIM, KERNEL, T>(i, g, pi, P, Q, R, E, n, I.G, I.K, nl, cnt, acc);
                else
#pragma unroll
                    for (int k = 0; k < 6; ++k) acc[k].zero();
                double a[3], xs[3];
                for (int d = 0; d < 3; ++d) {
                    a[d] = acc[d].value();
                    xs[d] = acc[3 + d].value();
                }
                momentum_finish<DIM>(i, fluid, a, xs, I.C, S, idt[inst], kick, mc);
            }
            if (cpart) {
                warp_mom_diag(mc);
                if (lane == 0) {
                    double* o = cpart + (size_t)c * 8;
                    o[0] = mc.px;
                    o[1] = mc.py;
                    o[2] = mc.pz;
                    o[3] = mc.ke;
                    o[4] = __longlong_as_double((long long)mc.u2b);
                    o[5] = __longlong_as_double((long long)mc.a2b);
                    o[6] = __longlong_as_double((long long)mc.bad);
                }
            }
        }
        return;
    }
    for (int tile = block; (long long)tile * GM < n; tile += nblocks) {
        const int i = tile * GM + grp;
        if (i < n) {
            const int inst = SINGLE ? 0 : find_instance(cell_bounds, ninst, skeys[i]);
            const Inst<Real>& I = SINGLE ? *I0 : tab[inst];
            const typename V4<Real>::T pi = P[i];
            const bool fluid = pi.w > Real(0);
            Acc<Real> acc[6];
            if (fluid) momentum_sums<Real, DIM, KERNEL, T>(i, g, pi, P, Q, R, E, n, I.G, I.K, nl, cnt, acc);
            else
#pragma unroll
                for (int k = 0; k < 6; ++k) acc[k].zero();
            if (T == 1) {
                double a[3], xs[3];
                for (int d = 0; d < 3; ++d) {
                    a[d] = acc[d].value();
                    xs[d] = acc[3 + d].value();
                }
                momentum_finish<DIM>(i, fluid, a, xs, I.C, S, idt[inst], kick, md);
            } else if (g.t == 0) {
#pragma unroll
                for (int k = 0; k < 6; ++k) {
                    sm.v[2 * k][grp] = acc[k].s;
                    sm.v[2 * k + 1][grp] = acc[k].c;
                }
                sm.fluid[grp] = fluid ? 1 : 0;
            }
        }
        if (T > 1) {
            __syncthreads();
            const int e = tile * GM + threadIdx.x;
            if (threadIdx.x < GM && e < n) {
                const int inst = SINGLE ? 0 : find_instance(cell_bounds, ninst, skeys[e]);
                double a[3], xs[3];
                for (int d = 0; d < 3; ++d) {
                    Acc<Real> x, y;
                    x.s = sm.v[2 * d][threadIdx.x];
                    x.c = sm.v[2 * d + 1][threadIdx.x];
                    y.s = sm.v[6 + 2 * d][threadIdx.x];
                    y.c = sm.v[6 + 2 * d + 1][threadIdx.x];
                    a[d] = x.value();
                    xs[d] = y.value();
                }
                momentum_finish<DIM>(e, sm.fluid[threadIdx.x] != 0, a, xs, SINGLE ? I0->C : tab[inst].C, S,
                                     idt[inst], kick, md);
            }
            __syncthreads();
        }
    }
}

// FP32: 8 blocks of 128 per SM in 2D (64 registers; the gathers of the pair loop are
// latency-bound and gain more from the extra warps than the few spills cost), 7 in 3D
// (72 registers: fewer spills of the longer 3D body measured faster); FP64: 5.
template <class Real, int DIM, int KERNEL, int T, bool SINGLE>
__global__ void __launch_bounds__(PAIR_THREADS, sizeof(Real) == 4 ? (DIM == 3 ? 7 : 8) : 5)
k_momentum(const __grid_constant__ Inst<Real> I0,
           const typename V4<Real>::T* __restrict__ P, const typename V4<Real>::T* __restrict__ Q,
           const Real* __restrict__ R, const F4* __restrict__ E, const uint32_t* __restrict__ skeys,
           int n,
           const Inst<Real>* __restrict__ tab, const uint32_t* __restrict__ cell_bounds, int ninst,
           double* __restrict__ idt, ParticleSet S, Control* ctl, int kick,
           const uint32_t* __restrict__ nl, const uint32_t* __restrict__ cnt,
           double* __restrict__ pm, const double* __restrict__ pd, int density_blocks,
           double* __restrict__ history, int finalize, double* __restrict__ cpart, int dyn) {
    constexpr int GM = PAIR_THREADS / T;
    __shared__ MomSmem<Real, T == 1 ? 1 : GM> sm;
    __shared__ MomDiag red[PAIR_THREADS / 32];
    __shared__ unsigned long long cred[PAIR_THREADS / 32][3];
    __shared__ bool is_last;
    if (ctl->status) return;
    MomDiag md{0, 0, 0, 0, 0ull, 0ull, 0u};
    // one lane per destination with dyn: chunks from a counter, for a batch (whose
    // diagnostics come from the state) or with chunk partials (cpart) for a single problem
    unsigned int* next = (T == 1 && dyn && (cpart != nullptr || !finalize)) ? &ctl->mom_next : nullptr;
    momentum_tiles<Real, DIM, KERNEL, T, PAIR_THREADS, SINGLE>(blockIdx.x, gridDim.x, P, Q, R, E, skeys, n,
                                                               tab, cell_bounds, ninst, idt, S, kick, nl, cnt,
                                                               md, sm, &I0, next, cpart);
    if (next) {  // the last block done resets the chunk counter for the next launch
        __syncthreads();
        if (threadIdx.x == 0) {
            const unsigned int d = atomicAdd(&ctl->mom_done, 1u);
            if (d == gridDim.x - 1) {
                ctl->mom_next = 0u;
                ctl->mom_done = 0u;
            }
        }
    }
    if (!finalize || cpart) return;  // chunk partials: k_mom_finalize reduces them
    const double dt = idt[0];
    // ---- block partials (epilogue threads: the first ceil(GM / 32) warps)
    block_mom_diag<(GM + 31) / 32>(md, pm + (size_t)blockIdx.x * 8, red);
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned t = atomicAdd(&ctl->ticket, 1u);
        is_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    // ---- last block: both passes' partials in a fixed order
    double out[10];
    reduce_partials<PAIR_THREADS>(pm, 8, gridDim.x, pd, 4, density_blocks, out, red, cred);
    if (threadIdx.x == 0) {
        ctl->ticket = 0;
        finish_single(ctl, history, SINGLE ? I0.C : tab[0].C, dt, kick, out);
    }
}

// Diagnostics of a single problem's evaluation whose momentum pass ran one lane per
// destination: block b sums the chunk partials of a fixed range of chunks (fixed order), the
// last block both passes' block partials, then writes the record, history entry, next dt and
// status. FIN_THREADS threads.
constexpr int FIN_THREADS = 256;

template <int NTH>
__global__ void __launch_bounds__(NTH)
k_mom_finalize(const double* __restrict__ cpart, int nchunks, double* __restrict__ pm,
               const double* __restrict__ pd, int density_blocks, Control* ctl,
               double* __restrict__ history, const StepConst C, const double* __restrict__ idt,
               int kick) {
    __shared__ MomDiag red[NTH / 32];
    __shared__ unsigned long long cred[NTH / 32][3];
    __shared__ bool is_last;
    if (ctl->status) return;
    const int per = (nchunks + gridDim.x - 1) / gridDim.x;
    const int lo = blockIdx.x * per, hi = min(nchunks, lo + per);
    MomDiag md{0, 0, 0, 0, 0ull, 0ull, 0u};
    for (int c = lo + threadIdx.x; c < hi; c += NTH) {
        const double* p = cpart + (size_t)c * 8;
        md.px += p[0];
        md.py += p[1];
        md.pz += p[2];
        md.ke += p[3];
        md.u2b = u64max(md.u2b, (unsigned long long)__double_as_longlong(p[4]));
        md.a2b = u64max(md.a2b, (unsigned long long)__double_as_longlong(p[5]));
        md.bad |= (unsigned)__double_as_longlong(p[6]);
    }
    block_mom_diag<NTH / 32>(md, pm + (size_t)blockIdx.x * 8, red);
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned t = atomicAdd(&ctl->ticket, 1u);
        is_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    double out[10];
    reduce_partials<NTH>(pm, 8, gridDim.x, pd, 4, density_blocks, out, red, cred);
    if (threadIdx.x == 0) {
        ctl->ticket = 0;
        finish_single(ctl, history, C, idt[0], kick, out);
    }
}

// ---------------------------------------------------------------- launchers
// Blocks per SM of each pass, in the single-problem or the batch form.
template <class Real, int DIM, int KERNEL, int T>
int density_bps(int single) {
    int b = 0;
    if (single) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_density<Real, DIM, KERNEL, T, true>, PAIR_THREADS, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_density<Real, DIM, KERNEL, T, false>, PAIR_THREADS, 0);
    return b > 0 ? b : 1;
}

template <class Real, int DIM, int KERNEL, int T>
int momentum_bps(int single) {
    int b = 0;
    if (single) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_momentum<Real, DIM, KERNEL, T, true>, PAIR_THREADS, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_momentum<Real, DIM, KERNEL, T, false>, PAIR_THREADS, 0);
    return b > 0 ? b : 1;
}

// A single problem (L.tab_host set) passes its constants by value; a batch its table.
template <class Real, int DIM, int KERNEL, int T>
void launch_density_t(const StepLaunch& L, cudaStream_t st) {
    using V = typename V4<Real>::T;
    const bool single = L.tab_host != nullptr;
    const Inst<Real> I0 = single ? *(const Inst<Real>*)L.tab_host : Inst<Real>{};
    auto k = single ? k_density<Real, DIM, KERNEL, T, true> : k_density<Real, DIM, KERNEL, T, false>;
    k<<<L.grid_d, PAIR_THREADS, 0, st>>>(
        I0, (const V*)L.P, (V*)L.Q, (Real*)L.R, (const F4*)L.E, L.skeys, L.off, L.n, (const Inst<Real>*)L.tab,
        L.cell_bounds, L.ninst, L.idt, L.S, L.ctl, L.kick, L.nl, L.cnt, L.maxn,
        L.finalize ? L.pd : nullptr, L.finalize ? nullptr : L.pcount, L.dyn);
}

template <class Real, int DIM, int KERNEL, int T>
void launch_momentum_t(const StepLaunch& L, cudaStream_t st) {
    using V = typename V4<Real>::T;
    const bool single = L.tab_host != nullptr;
    const Inst<Real> I0 = single ? *(const Inst<Real>*)L.tab_host : Inst<Real>{};
    auto k = single ? k_momentum<Real, DIM, KERNEL, T, true> : k_momentum<Real, DIM, KERNEL, T, false>;
    // chunks taken from a counter where costs differ widely (wall destinations have no pair
    // sums); a single problem's diagnostics then go through chunk partials and k_mom_finalize
    const bool dyn = T == 1 && (L.dyn & 2);
    const bool chunked = dyn && L.finalize && single && L.cpart;
    k<<<L.grid_m, PAIR_THREADS, 0, st>>>(
        I0, (const V*)L.P, (const V*)L.Q, (const Real*)L.R, (const F4*)L.E, L.skeys, L.n,
        (const Inst<Real>*)L.tab, L.cell_bounds, L.ninst, L.idt, L.S, L.ctl, L.kick, L.nl, L.cnt, L.pm, L.pd,
        L.grid_d, L.history, L.finalize, chunked ? L.cpart : nullptr, dyn ? 1 : 0);
    if (chunked) {
        const int nchunks = (L.n + MOM_CHUNK - 1) / MOM_CHUNK;
        int nb = (nchunks + FIN_THREADS - 1) / FIN_THREADS;
        nb = nb < 1 ? 1 : (nb > L.sms ? L.sms : nb);
        const StepConst C = single ? I0.C : StepConst{};
        k_mom_finalize<FIN_THREADS><<<nb, FIN_THREADS, 0, st>>>(L.cpart, nchunks, L.pm, L.pd, L.grid_d, L.ctl, L.history, C,
                                                  L.idt, L.kick);
    }
}

// One precision's dispatch over (dim, kernel, group size).
template <class Real>
struct PairDispatch {
    template <int T>
    static int bps_t(int pass, int dim, int kernel, int single) {
        const int sel = (dim == 3 ? 3 : 0) + kernel;
        switch (sel) {
            case 0: return pass ? momentum_bps<Real, 2, QUINTIC, T>(single) : density_bps<Real, 2, QUINTIC, T>(single);
            case 1: return pass ? momentum_bps<Real, 2, WENDLAND_C2, T>(single) : density_bps<Real, 2, WENDLAND_C2, T>(single);
            case 2: return pass ? momentum_bps<Real, 2, CUBIC_SPLINE, T>(single) : density_bps<Real, 2, CUBIC_SPLINE, T>(single);
            case 3: return pass ? momentum_bps<Real, 3, QUINTIC, T>(single) : density_bps<Real, 3, QUINTIC, T>(single);
            case 4: return pass ? momentum_bps<Real, 3, WENDLAND_C2, T>(single) : density_bps<Real, 3, WENDLAND_C2, T>(single);
            default: return pass ? momentum_bps<Real, 3, CUBIC_SPLINE, T>(single) : density_bps<Real, 3, CUBIC_SPLINE, T>(single);
        }
    }
    template <int T>
    static void density_t(const StepLaunch& L, cudaStream_t st) {
        const int sel = (L.dim == 3 ? 3 : 0) + L.kernel;
        switch (sel) {
            case 0: launch_density_t<Real, 2, QUINTIC, T>(L, st); break;
            case 1: launch_density_t<Real, 2, WENDLAND_C2, T>(L, st); break;
            case 2: launch_density_t<Real, 2, CUBIC_SPLINE, T>(L, st); break;
            case 3: launch_density_t<Real, 3, QUINTIC, T>(L, st); break;
            case 4: launch_density_t<Real, 3, WENDLAND_C2, T>(L, st); break;
            default: launch_density_t<Real, 3, CUBIC_SPLINE, T>(L, st); break;
        }
    }
    template <int T>
    static void momentum_t(const StepLaunch& L, cudaStream_t st) {
        const int sel = (L.dim == 3 ? 3 : 0) + L.kernel;
        switch (sel) {
            case 0: launch_momentum_t<Real, 2, QUINTIC, T>(L, st); break;
            case 1: launch_momentum_t<Real, 2, WENDLAND_C2, T>(L, st); break;
            case 2: launch_momentum_t<Real, 2, CUBIC_SPLINE, T>(L, st); break;
            case 3: launch_momentum_t<Real, 3, QUINTIC, T>(L, st); break;
            case 4: launch_momentum_t<Real, 3, WENDLAND_C2, T>(L, st); break;
            default: launch_momentum_t<Real, 3, CUBIC_SPLINE, T>(L, st); break;
        }
    }
};

template <class Real, int T>
int pair_bps(int pass, int dim, int kernel, int single) {
    return PairDispatch<Real>::template bps_t<T>(pass, dim, kernel, single);
}
template <class Real, int T>
void pair_density(const StepLaunch& L, cudaStream_t st) {
    PairDispatch<Real>::template density_t<T>(L, st);
}
template <class Real, int T>
void pair_momentum(const StepLaunch& L, cudaStream_t st) {
    PairDispatch<Real>::template momentum_t<T>(L, st);
}

}  // namespace sph
