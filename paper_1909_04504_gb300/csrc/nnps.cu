// Neighbour-search build of the uniform cell grid (Sec. 2.2, the Z-order / cell-sort
// approach the paper provides on GPUs): cell key per particle (fused with the
// predictor half-kick and drift of Sec. 2.1 and the periodic wrap), a stable LSD radix
// sort of (key, index), the gather of the FP64 state into cell order with the Tait EOS
// (Eq. eos) fused into the write of the pair-loop shadow arrays, and the cell table.
#include "sph_device.cuh"
#include "sph_launch.h"
#include "sort_impl.cuh"
#include "step_impl.cuh"
#include "stencil.cuh"

namespace sph {

// ----------------------------------------------------------- drift + cell key
// Per particle in the current order: for fluid, u_half = u + dt/2 a and
// x <- wrap(x + dt (u_half + xsph)) (written back in place); then the linear cell id
// of the position rounded to the pair-loop precision.
template <class Real>
__global__ void k_drift_keys(ParticleSet S, int n, const Inst<Real>* __restrict__ tab,
                             const uint32_t* __restrict__ id_bounds, int ninst,
                             const double* __restrict__ idt, int drift, uint32_t* keys,
                             Control* ctl) {
    if (ctl->status) return;
    unsigned outside = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int inst = find_instance(id_bounds, ninst, S.tag[i] & ID_MASK);
        const Inst<Real>& I = tab[inst];
        int clamped = 0;
        keys[i] = I.cell_base + drift_key_one(S, i, I.G, I.C, idt[inst], drift, clamped);
        outside += clamped;
    }
    // count clamped particles (warp-aggregated)
    for (int o = 16; o > 0; o >>= 1) outside += __shfl_down_sync(0xffffffffu, outside, o);
    if ((threadIdx.x & 31) == 0 && outside) atomicAdd(&ctl->outside, outside);
}

// Drift + cell key as above, and the digit histograms of all radix passes of the keys
// (block histograms in shared memory, added to ghist[pass * 256 + digit]). 256 threads.
template <class Real>
__global__ void __launch_bounds__(256)
k_keys_hist(ParticleSet S, int n, const Inst<Real>* __restrict__ tab,
            const uint32_t* __restrict__ id_bounds, int ninst, const double* __restrict__ idt,
            int drift, uint32_t* keys, uint32_t* __restrict__ ghist, int passes, Control* ctl) {
    __shared__ uint32_t h[4][RADIX];
    if (ctl->status) return;
    for (int p = 0; p < passes; ++p) h[p][threadIdx.x] = 0;
    __syncthreads();
    unsigned outside = 0;
    for (int base = blockIdx.x * 256; base < n; base += gridDim.x * 256) {
        const int i = base + threadIdx.x;
        const bool valid = i < n;
        uint32_t key = 0;
        if (valid) {
            const int inst = find_instance(id_bounds, ninst, S.tag[i] & ID_MASK);
            const Inst<Real>& I = tab[inst];
            int clamped = 0;
            key = I.cell_base + drift_key_one(S, i, I.G, I.C, idt[inst], drift, clamped);
            keys[i] = key;
            outside += clamped;
        }
        digit_hist_add(key, valid, passes, h);
    }
    for (int o = 16; o > 0; o >>= 1) outside += __shfl_down_sync(0xffffffffu, outside, o);
    if ((threadIdx.x & 31) == 0 && outside) atomicAdd(&ctl->outside, outside);
    __syncthreads();
    for (int p = 0; p < passes; ++p) {
        const uint32_t v = h[p][threadIdx.x];
        if (v) atomicAdd(&ghist[p * RADIX + threadIdx.x], v);
    }
}

// One radix pass in one launch (decoupled look-back); one tile per block. Tiles of 8 keys
// per thread are held to 48 registers (5 blocks per SM instead of 4 at 60: 2 % faster on
// 2.9 M keys; tiles of 16 keys were slower at either occupancy), tiles of 4 to 40.
template <int ITEMS>
__global__ void __launch_bounds__(SORT_THREADS, ITEMS == 8 ? 5 : 6)
k_radix_onesweep(const uint32_t* __restrict__ keys_in, const uint32_t* __restrict__ vals_in,
                 uint32_t* __restrict__ keys_out, uint32_t* __restrict__ vals_out, int n, int shift,
                 const uint32_t* __restrict__ ghist, uint32_t* status, uint32_t* counter,
                 Control* ctl, unsigned long long wait_ns) {
    __shared__ OnesweepSmem sm;
    if (ctl->status) return;
    if (threadIdx.x == 0) sm.tile = (int)atomicAdd(counter, 1u);
    __syncthreads();
    radix_onesweep_tile<ITEMS>(keys_in, vals_in, keys_out, vals_out, n, shift, ghist, status,
                               sm.tile, sm, &ctl->status, wait_ns);
}

// -------------------------------------------------------------- radix sort
// Block bodies in sort_impl.cuh (shared with the persistent step kernel).
__global__ void __launch_bounds__(SORT_THREADS)
k_radix_hist(const uint32_t* __restrict__ keys, int n, int shift, uint32_t* hist, int nblocks,
             const Control* ctl) {
    __shared__ uint32_t h[RADIX];
    if (ctl->status) return;
    radix_hist_tile(keys, n, shift, hist, nblocks, blockIdx.x, h);
}

__global__ void __launch_bounds__(1024)
k_radix_scan(uint32_t* hist, int nblocks, uint32_t* totals, const Control* ctl) {
    __shared__ uint32_t wsum[32];
    if (ctl->status) return;
    radix_scan_row(hist, nblocks, totals, blockIdx.x, wsum);
}

__global__ void __launch_bounds__(SORT_THREADS)
k_radix_scatter(const uint32_t* __restrict__ keys_in, const uint32_t* __restrict__ vals_in,
                uint32_t* __restrict__ keys_out, uint32_t* __restrict__ vals_out, int n, int shift,
                const uint32_t* __restrict__ hist, const uint32_t* __restrict__ totals, int nblocks,
                const Control* ctl) {
    __shared__ ScatterSmem sm;
    if (ctl->status) return;
    radix_scatter_tile(keys_in, vals_in, keys_out, vals_out, n, shift, hist, totals, nblocks,
                       blockIdx.x, sm);
}

// offsets[c] = number of sorted keys < c, for c in [0, ncells].
__global__ void k_cell_offsets(const uint32_t* __restrict__ skeys, int n, int ncells,
                               uint32_t* __restrict__ off, const Control* ctl) {
    if (ctl->status) return;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c <= ncells; c += gridDim.x * blockDim.x)
        off[c] = cell_offset(skeys, n, (uint32_t)c);
}

// ------------------------------------------------------------------ reorder
// Gather the state into cell order. kick: predictor half-kick of the fluid velocity
// (the density is advanced later, like the positions, by the density pass). Rates are
// carried along only outside a step (carry_rates).
// Writes the pair-loop shadow: P = (x, y, z, +-m) with the sign marking walls,
// Q = (u, v, w, rho), R = p / rho^2 with p from the Tait EOS (Eq. eos) in FP64.
template <class Real>
__global__ void k_reorder(ParticleSet in, ParticleSet out, const uint32_t* __restrict__ perm,
                          const uint32_t* __restrict__ skeys, int n, int dim,
                          const Inst<Real>* __restrict__ tab, const uint32_t* __restrict__ cell_bounds,
                          int ninst, const double* __restrict__ idt, int kick, int carry_rates,
                          typename V4<Real>::T* __restrict__ P, typename V4<Real>::T* __restrict__ Q,
                          F4* __restrict__ E, int edac, uint32_t* __restrict__ off, int ncells,
                          uint32_t* __restrict__ work, int work_words, const Control* ctl) {
    if (ctl->status) return;
    // cell table: four consecutive cells per thread, their previous offsets read and the
    // new ones written as one 16-byte word (grids with many more cells than particles,
    // as the half-size cells of 3D, would otherwise take several loop trips per thread);
    // the sort passes are done, so their workspace (histograms, tile counters, look-back
    // words) is cleared here for the next build instead of by a separate memset
    const int nq = (ncells + 4) / 4;
    int m = n > nq ? n : nq;
    m = m > work_words ? m : work_words;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x) {
        if (k < work_words) work[k] = 0u;
        if (k < n) {
            const int inst = find_instance(cell_bounds, ninst, skeys[k]);
            reorder_one<Real>(in, out, k, (int)perm[k], dim, idt[inst], kick, carry_rates, P, Q, E,
                              edac);
        }
        if (k < nq) {
            const uint32_t c0 = 4u * (uint32_t)k;
            if (c0 + 3 <= (uint32_t)ncells) {
                uint4 g = reinterpret_cast<const uint4*>(off)[k];
                g.x = cell_offset_near(skeys, n, c0, g.x);
                g.y = cell_offset_near(skeys, n, c0 + 1, g.y);
                g.z = cell_offset_near(skeys, n, c0 + 2, g.z);
                g.w = cell_offset_near(skeys, n, c0 + 3, g.w);
                reinterpret_cast<uint4*>(off)[k] = g;
            } else {
                for (uint32_t c = c0; c <= (uint32_t)ncells; ++c) off[c] = cell_offset_near(skeys, n, c, off[c]);
            }
        }
    }
}

// --------------------------------------------------------- get / set helpers
// out[id - first] = field[k] for particles whose global id lies in [first, first + count).
__global__ void k_gather_by_id(const double* __restrict__ field, const uint32_t* __restrict__ tag,
                               int n, uint32_t first, uint32_t count, double* __restrict__ out) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        uint32_t id = tag[k] & ID_MASK;
        if (id - first < count) out[id - first] = field[k];
    }
}

__global__ void k_scatter_by_id(double* __restrict__ field, const uint32_t* __restrict__ tag, int n,
                                uint32_t first, uint32_t count, const double* __restrict__ in) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        uint32_t id = tag[k] & ID_MASK;
        if (id - first < count) field[k] = in[id - first];
    }
}

__global__ void k_cell_of_by_id(const uint32_t* __restrict__ skeys, const uint32_t* __restrict__ tag,
                                int n, uint32_t* __restrict__ cell_of, int64_t* __restrict__ order) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        uint32_t id = tag[k] & ID_MASK;
        cell_of[id] = skeys[k];
        order[k] = (int64_t)id;
    }
}

// Wrap periodic coordinates into the box (at creation and after sph_set).
__global__ void k_wrap_all(ParticleSet S, int n, Grid G) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        for (int d = 0; d < G.dim; ++d) {
            if (!G.periodic[d]) continue;
            double x = S.x[d][i];
            if (x >= G.lo[d] && x < G.hi[d]) continue;
            double k = floor(__ddiv_rn(__dsub_rn(x, G.lo[d]), G.L[d]));
            x = __dsub_rn(x, __dmul_rn(k, G.L[d]));
            if (x >= G.hi[d]) x = __dsub_rn(x, G.L[d]);
            if (x < G.lo[d]) x = G.lo[d];
            S.x[d][i] = x;
        }
    }
}

// ------------------------------------------------------ neighbour export
// The same stencil walk and predicate as the pair loops; pass 0 counts, pass 1 writes
// the original ids of the neighbours of sorted particle k at offsets[id(k)] and sorts
// the row ascending.
template <class Real, int DIM>
__global__ void k_export_neighbors(const typename V4<Real>::T* __restrict__ P,
                                   const uint32_t* __restrict__ skeys,
                                   const uint32_t* __restrict__ off,
                                   const uint32_t* __restrict__ tag, int n, Grid G,
                                   PairConst<Real> K, int pass, uint32_t* __restrict__ counts,
                                   const int64_t* __restrict__ row_off, int32_t* __restrict__ idx) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const typename V4<Real>::T pi = P[i];
        int cx, cy, cz;
        cell_of_key(G, skeys[i], cx, cy, cz);
        const uint32_t id = tag[i] & ID_MASK;
        int64_t w = pass ? row_off[id] : 0;
        const int64_t w0 = w;
        uint32_t cnt = 0;
        for_each_run<DIM>(G, off, cx, cy, cz, [&](uint32_t jb, uint32_t je) {
            for (uint32_t j = jb; j < je; ++j) {
                if ((int)j == i) continue;
                const typename V4<Real>::T pj = P[j];
                const Real dx = min_image(rn_sub(pi.x, pj.x), G.periodic[0], K.L[0], K.halfL[0]);
                const Real dy = min_image(rn_sub(pi.y, pj.y), G.periodic[1], K.L[1], K.halfL[1]);
                const Real dzv = DIM == 3 ? min_image(rn_sub(pi.z, pj.z), G.periodic[2], K.L[2], K.halfL[2])
                                          : Real(0);
                const Real r2 = dist2<Real, DIM>(dx, dy, dzv);
                if (!(r2 < K.kh2)) continue;
                if (pass) idx[w++] = (int32_t)(tag[j] & ID_MASK);
                ++cnt;
            }
        });
        if (!pass) {
            counts[id] = cnt;
        } else {
            for (int64_t a = w0 + 1; a < w; ++a) {  // insertion sort of the row
                const int32_t v = idx[a];
                int64_t b = a - 1;
                while (b >= w0 && idx[b] > v) { idx[b + 1] = idx[b]; --b; }
                idx[b + 1] = v;
            }
        }
    }
}

// ---------------------------------------------------------------- launchers
static inline int grid_for(long long n, int threads, int cap) {
    long long b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (int)b;
}

void launch_drift_keys(const StepLaunch& L, int drift, uint32_t* keys, cudaStream_t st) {
    const int g = grid_for(L.n, 256, L.sms * 8);
    if (L.precision)
        k_drift_keys<float><<<g, 256, 0, st>>>(L.Sin, L.n, (const Inst<float>*)L.tab, L.id_bounds,
                                               L.ninst, L.idt, drift, keys, L.ctl);
    else
        k_drift_keys<double><<<g, 256, 0, st>>>(L.Sin, L.n, (const Inst<double>*)L.tab, L.id_bounds,
                                                L.ninst, L.idt, drift, keys, L.ctl);
}

int radix_passes(int ncells) {
    int bits = 0;
    while (bits < 32 && (1ull << bits) < (unsigned long long)ncells) ++bits;
    return (bits + 7) / 8;
}

int radix_tiles(int n) {
    const int t = (n + SORT_TILE - 1) / SORT_TILE;
    return t < 1 ? 1 : t;
}

size_t radix_hist_words(int n) { return radix_hist_words_for(n); }

// Sorts (keys[0], iota) by the low `passes * 8` bits; returns the buffer index (0 or 1)
// holding the sorted keys and the permutation (sorted position -> previous position).
int launch_radix_sort(uint32_t* keys[2], uint32_t* vals[2], int n, int passes, uint32_t* hist,
                      Control* ctl, cudaStream_t st) {
    int nblocks = (n + SORT_TILE - 1) / SORT_TILE;
    if (nblocks < 1) nblocks = 1;
    uint32_t* totals = hist + (size_t)RADIX * nblocks;
    int cur = 0;
    for (int p = 0; p < passes; ++p) {
        int shift = 8 * p;
        k_radix_hist<<<nblocks, SORT_THREADS, 0, st>>>(keys[cur], n, shift, hist, nblocks, ctl);
        k_radix_scan<<<RADIX, 1024, 0, st>>>(hist, nblocks, totals, ctl);
        k_radix_scatter<<<nblocks, SORT_THREADS, 0, st>>>(keys[cur], p == 0 ? nullptr : vals[cur],
                                                          keys[cur ^ 1], vals[cur ^ 1], n, shift,
                                                          hist, totals, nblocks, ctl);
        cur ^= 1;
    }
    return cur;
}

void launch_cell_offsets(const uint32_t* skeys, int n, int ncells, uint32_t* off, Control* ctl,
                         cudaStream_t st, int sms) {
    k_cell_offsets<<<grid_for((long long)ncells + 1, 256, sms * 8), 256, 0, st>>>(skeys, n, ncells,
                                                                                  off, ctl);
}

void launch_reorder(const StepLaunch& L, const uint32_t* perm, int carry_rates, uint32_t* off,
                    int ncells, uint32_t* work, int work_words, cudaStream_t st) {
    const int nq = (ncells + 4) / 4;
    int m = L.n > nq ? L.n : nq;
    m = m > work_words ? m : work_words;
    const int g = grid_for(m, 256, L.sms * 8);
    if (L.precision)
        k_reorder<float><<<g, 256, 0, st>>>(L.Sin, L.S, perm, L.skeys, L.n, L.dim,
                                            (const Inst<float>*)L.tab, L.cell_bounds, L.ninst, L.idt,
                                            L.kick, carry_rates, (F4*)L.P, (F4*)L.Q, (F4*)L.E, L.edac,
                                            off, ncells, work, work_words, L.ctl);
    else
        k_reorder<double><<<g, 256, 0, st>>>(L.Sin, L.S, perm, L.skeys, L.n, L.dim,
                                             (const Inst<double>*)L.tab, L.cell_bounds, L.ninst,
                                             L.idt, L.kick, carry_rates, (D4*)L.P, (D4*)L.Q, nullptr,
                                             L.edac, off, ncells, work, work_words, L.ctl);
}

size_t sort_work_words(int n, int passes) {
    return (size_t)4 * RADIX + 32 + (size_t)passes * onesweep_tiles(n) * RADIX;
}

// Zeroes the sort workspace, then drift + keys + the digit histograms of all passes.
void launch_keys_hist(const StepLaunch& L, int drift, uint32_t* keys0, int passes, uint32_t* work,
                      cudaStream_t st) {
    const int g = grid_for(L.n, 256, L.sms * 8);
    if (L.precision)
        k_keys_hist<float><<<g, 256, 0, st>>>(L.Sin, L.n, (const Inst<float>*)L.tab, L.id_bounds,
                                              L.ninst, L.idt, drift, keys0, work, passes, L.ctl);
    else
        k_keys_hist<double><<<g, 256, 0, st>>>(L.Sin, L.n, (const Inst<double>*)L.tab, L.id_bounds,
                                               L.ninst, L.idt, drift, keys0, work, passes, L.ctl);
}

// One one-sweep launch per pass over (keys[0], identity). Returns the buffer index (0 or
// 1) holding the sorted keys and the permutation.
int launch_onesweep(int n, uint32_t* keys[2], uint32_t* vals[2], int passes, uint32_t* work,
                    Control* ctl, unsigned long long wait_ns, cudaStream_t st) {
    const int ntiles = onesweep_tiles(n);
    uint32_t* ghist = work;
    uint32_t* counters = work + 4 * RADIX;
    uint32_t* status = counters + 32;
    int cur = 0;
    for (int p = 0; p < passes; ++p) {
        const uint32_t* vin = p == 0 ? nullptr : vals[cur];
        uint32_t* st_p = status + (size_t)p * ntiles * RADIX;
        switch (onesweep_items(n)) {
            case 4:
                k_radix_onesweep<4><<<ntiles, SORT_THREADS, 0, st>>>(
                    keys[cur], vin, keys[cur ^ 1], vals[cur ^ 1], n, 8 * p, ghist + p * RADIX,
                    st_p, counters + p, ctl, wait_ns);
                break;
            default:
                k_radix_onesweep<8><<<ntiles, SORT_THREADS, 0, st>>>(
                    keys[cur], vin, keys[cur ^ 1], vals[cur ^ 1], n, 8 * p, ghist + p * RADIX,
                    st_p, counters + p, ctl, wait_ns);
                break;
        }
        cur ^= 1;
    }
    return cur;
}

void launch_gather_by_id(const double* field, const uint32_t* tag, int n, uint32_t first,
                         uint32_t count, double* out, cudaStream_t st, int sms) {
    k_gather_by_id<<<grid_for(n, 256, sms * 8), 256, 0, st>>>(field, tag, n, first, count, out);
}

void launch_scatter_by_id(double* field, const uint32_t* tag, int n, uint32_t first,
                          uint32_t count, const double* in, cudaStream_t st, int sms) {
    k_scatter_by_id<<<grid_for(n, 256, sms * 8), 256, 0, st>>>(field, tag, n, first, count, in);
}

void launch_cell_of_by_id(const uint32_t* skeys, const uint32_t* tag, int n, uint32_t* cell_of,
                          int64_t* order, cudaStream_t st, int sms) {
    k_cell_of_by_id<<<grid_for(n, 256, sms * 8), 256, 0, st>>>(skeys, tag, n, cell_of, order);
}

void launch_wrap_all(const ParticleSet& S, int n, const Grid& G, cudaStream_t st, int sms) {
    k_wrap_all<<<grid_for(n, 256, sms * 8), 256, 0, st>>>(S, n, G);
}

void launch_export_neighbors(int precision, int dim, const void* P, const uint32_t* skeys,
                             const uint32_t* off, const uint32_t* tag, int n, const Grid& G,
                             const PairConst<float>& Kf, const PairConst<double>& Kd, int pass,
                             uint32_t* counts, const int64_t* row_off, int32_t* idx,
                             cudaStream_t st, int sms) {
    int g = grid_for(n, 128, sms * 16);
    if (precision) {
        if (dim == 2)
            k_export_neighbors<float, 2><<<g, 128, 0, st>>>((const F4*)P, skeys, off, tag, n, G, Kf,
                                                            pass, counts, row_off, idx);
        else
            k_export_neighbors<float, 3><<<g, 128, 0, st>>>((const F4*)P, skeys, off, tag, n, G, Kf,
                                                            pass, counts, row_off, idx);
    } else {
        if (dim == 2)
            k_export_neighbors<double, 2><<<g, 128, 0, st>>>((const D4*)P, skeys, off, tag, n, G, Kd,
                                                             pass, counts, row_off, idx);
        else
            k_export_neighbors<double, 3><<<g, 128, 0, st>>>((const D4*)P, skeys, off, tag, n, G, Kd,
                                                             pass, counts, row_off, idx);
    }
}

}  // namespace sph
