// Block-level bodies of the stable LSD radix sort (8-bit digits) of the cell keys and of
// the cell table (Sec. 2.2 cell-sort neighbour search), shared by the per-phase kernels
// and the persistent step kernel. A tile of SORT_TILE keys belongs to one block; inside
// the tile warp w owns the contiguous range [w * 512, (w + 1) * 512) and walks it in
// order, so tile order, warp order, iteration order and lane order reproduce the input
// order (stability).
#pragma once

#include "sph_device.cuh"

namespace sph {

constexpr int RADIX = 256;
constexpr int SORT_THREADS = 256;
constexpr int SORT_WARPS = SORT_THREADS / 32;
constexpr int SORT_ITEMS = 16;
constexpr int SORT_TILE = SORT_THREADS * SORT_ITEMS;

// Words of the digit histograms of launch_radix_sort for n keys: RADIX counts per tile of
// SORT_TILE keys, then the RADIX digit totals.
constexpr size_t radix_hist_words_for(long long n) {
    return (size_t)RADIX * (size_t)(n > 0 ? (n + SORT_TILE - 1) / SORT_TILE : 1) + RADIX;
}

struct ScatterSmem {
    uint32_t base_d[RADIX];
    uint32_t wcnt[SORT_WARPS][RADIX];
    uint32_t wsum[SORT_WARPS];
};

// Digit histogram of tile `tile` into hist[digit * ntiles + tile] (SORT_THREADS threads).
__device__ __forceinline__ void radix_hist_tile(const uint32_t* __restrict__ keys, int n, int shift,
                                                uint32_t* __restrict__ hist, int ntiles, int tile,
                                                uint32_t* h) {
    h[threadIdx.x] = 0;
    __syncthreads();
    const int base = tile * SORT_TILE;
#pragma unroll 4
    for (int k = 0; k < SORT_ITEMS; ++k) {
        const int idx = base + k * SORT_THREADS + threadIdx.x;
        if (idx < n) atomicAdd(&h[(keys[idx] >> shift) & (RADIX - 1)], 1u);
    }
    __syncthreads();
    hist[threadIdx.x * ntiles + tile] = h[threadIdx.x];
}

// Exclusive scan of digit `digit`'s row of per-tile counts; totals[digit] = row sum.
// Any block size that is a multiple of 32 (up to 1024).
__device__ __forceinline__ void radix_scan_row(uint32_t* __restrict__ hist, int ntiles,
                                               uint32_t* __restrict__ totals, int digit,
                                               uint32_t* wsum) {
    uint32_t* row = hist + (size_t)digit * ntiles;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t carry = 0;
    for (int base = 0; base < ntiles; base += blockDim.x) {
        const int i = base + threadIdx.x;
        const uint32_t v = i < ntiles ? row[i] : 0u;
        uint32_t x = v;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[warp] = x;
        __syncthreads();
        if (warp == 0) {
            uint32_t s = lane < nw ? wsum[lane] : 0u;
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
                if (lane >= o) s += y;
            }
            wsum[lane] = s;
        }
        __syncthreads();
        const uint32_t excl = carry + x - v + (warp ? wsum[warp - 1] : 0u);
        if (i < ntiles) row[i] = excl;
        carry += wsum[nw - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0) totals[digit] = carry;
}

// Stable scatter of tile `tile` (SORT_THREADS threads): digit base = exclusive scan of the
// digit totals + this tile's offset in its digit row; rank inside the tile by per-warp
// match_any counting in warp order. vals_in == nullptr: the values are the input indices.
__device__ __forceinline__ void radix_scatter_tile(const uint32_t* __restrict__ keys_in,
                                                   const uint32_t* __restrict__ vals_in,
                                                   uint32_t* __restrict__ keys_out,
                                                   uint32_t* __restrict__ vals_out, int n, int shift,
                                                   const uint32_t* __restrict__ hist,
                                                   const uint32_t* __restrict__ totals, int ntiles,
                                                   int tile, ScatterSmem& sm) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    {
        const uint32_t v = totals[tid];
        uint32_t x = v;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) sm.wsum[warp] = x;
        for (int w = 0; w < SORT_WARPS; ++w) sm.wcnt[w][tid] = 0;
        __syncthreads();
        uint32_t pre = 0;
        for (int w = 0; w < warp; ++w) pre += sm.wsum[w];
        sm.base_d[tid] = pre + x - v + hist[tid * ntiles + tile];
    }
    __syncthreads();
    const int wbase = tile * SORT_TILE + warp * (SORT_TILE / SORT_WARPS);
    uint32_t kr[SORT_ITEMS], vr[SORT_ITEMS], rank[SORT_ITEMS];
    const unsigned ltmask = lanemask_lt();
#pragma unroll
    for (int it = 0; it < SORT_ITEMS; ++it) {
        const int idx = wbase + it * 32 + lane;
        const bool valid = idx < n;
        const uint32_t key = valid ? keys_in[idx] : 0u;
        const uint32_t d = valid ? ((key >> shift) & (RADIX - 1)) : (uint32_t)RADIX;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const uint32_t before = valid ? sm.wcnt[warp][d] : 0u;
        __syncwarp();
        if (valid && lane == __ffs(peers) - 1) sm.wcnt[warp][d] = before + __popc(peers);
        __syncwarp();
        kr[it] = key;
        vr[it] = valid ? (vals_in ? vals_in[idx] : (uint32_t)idx) : 0u;
        rank[it] = before + __popc(peers & ltmask);
    }
    __syncthreads();
    {   // exclusive prefix over warps, per digit
        uint32_t run = 0;
        for (int w = 0; w < SORT_WARPS; ++w) {
            const uint32_t c = sm.wcnt[w][tid];
            sm.wcnt[w][tid] = run;
            run += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < SORT_ITEMS; ++it) {
        const int idx = wbase + it * 32 + lane;
        if (idx < n) {
            const uint32_t d = (kr[it] >> shift) & (RADIX - 1);
            const uint32_t pos = sm.base_d[d] + sm.wcnt[warp][d] + rank[it];
            keys_out[pos] = kr[it];
            vals_out[pos] = vr[it];
        }
    }
}

// ------------------------------------------------------------ one-sweep passes
// A pass in one launch: every tile ranks its keys locally, publishes its per-digit count
// and looks back over the preceding tiles' published counts for its exclusive prefix
// (decoupled look-back), while the global digit bases come from a histogram of all passes
// taken beforehand (with the cell keys). Tiles take their index from a counter in launch
// order, so every tile a tile waits for has started and waits only on earlier tiles.
// Status word per (tile, digit): 2 flag bits (aggregate / inclusive prefix) + 30-bit count.
// The tile is put in digit order in shared memory before the look-back, and written out
// from there in that order: a warp's 32 stores then cover a few runs of consecutive
// positions instead of up to 32 scattered words.
constexpr uint32_t LB_AGGREGATE = 1u << 30;
constexpr uint32_t LB_PREFIX = 2u << 30;
constexpr uint32_t LB_COUNT = (1u << 30) - 1u;
// Predecessors read per look-back round (32 measured slower than 8 on 2.9 M keys: the
// rounds are not what bounds a pass).
constexpr int LB_BATCH = 8;
constexpr int ONESWEEP_MAX_ITEMS = 8;

struct OnesweepSmem {
    uint32_t base_d[RADIX];
    uint32_t wcnt[SORT_WARPS][RADIX];
    uint32_t wsum[SORT_WARPS];
    uint32_t sk[SORT_THREADS * ONESWEEP_MAX_ITEMS];  // the tile in digit order
    uint32_t sv[SORT_THREADS * ONESWEEP_MAX_ITEMS];
    int tile;
};

__device__ __forceinline__ unsigned long long sort_clock_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Keys per thread of a one-sweep tile: small problems take short tiles (more blocks,
// shorter serial ranking loops), large ones tiles of 2,048 keys.
__host__ __device__ __forceinline__ int onesweep_items(int n) { return n <= 131072 ? 4 : 8; }
__host__ __device__ __forceinline__ int onesweep_tiles(int n) {
    const int tile = SORT_THREADS * onesweep_items(n);
    const int t = (n + tile - 1) / tile;
    return t < 1 ? 1 : t;
}

// Exclusive scan of v over the block's SORT_THREADS threads (thread tid holds digit tid).
// Uses wsum: the caller separates two calls by a barrier.
__device__ __forceinline__ uint32_t digit_scan_excl(uint32_t v, uint32_t* wsum) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    uint32_t pre = 0;
    for (int w = 0; w < warp; ++w) pre += wsum[w];
    return pre + x - v;
}

// One tile of a one-sweep pass (SORT_THREADS threads, ITEMS keys each). ghist: the RADIX
// digit counts of this pass over all keys; status: ntiles x RADIX look-back words, zero
// before the pass. A look-back wait longer than wait_ns raises ST_TIMEOUT and the tile
// writes nothing.
template <int ITEMS>
__device__ __forceinline__ void radix_onesweep_tile(const uint32_t* __restrict__ keys_in,
                                                    const uint32_t* __restrict__ vals_in,
                                                    uint32_t* __restrict__ keys_out,
                                                    uint32_t* __restrict__ vals_out, int n,
                                                    int shift, const uint32_t* __restrict__ ghist,
                                                    uint32_t* status, int tile,
                                                    OnesweepSmem& sm, unsigned* ctl_status,
                                                    unsigned long long wait_ns) {
    static_assert(ITEMS <= ONESWEEP_MAX_ITEMS, "tile larger than its shared staging");
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int w = 0; w < SORT_WARPS; ++w) sm.wcnt[w][tid] = 0;
    __syncthreads();
    constexpr int TILE = SORT_THREADS * ITEMS;
    const int wbase = tile * TILE + warp * (TILE / SORT_WARPS);
    uint32_t kr[ITEMS], vr[ITEMS], rank[ITEMS];
    const unsigned ltmask = lanemask_lt();
    // ranks inside the warp's contiguous range, in input order (stability)
#pragma unroll
    for (int it = 0; it < ITEMS; ++it) {
        const int idx = wbase + it * 32 + lane;
        const bool valid = idx < n;
        const uint32_t key = valid ? keys_in[idx] : 0u;
        const uint32_t d = valid ? ((key >> shift) & (RADIX - 1)) : (uint32_t)RADIX;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const uint32_t before = valid ? sm.wcnt[warp][d] : 0u;
        __syncwarp();
        if (valid && lane == __ffs(peers) - 1) sm.wcnt[warp][d] = before + __popc(peers);
        __syncwarp();
        kr[it] = key;
        vr[it] = valid ? (vals_in ? vals_in[idx] : (uint32_t)idx) : 0u;
        rank[it] = before + __popc(peers & ltmask);
    }
    __syncthreads();
    // per digit (thread tid): exclusive prefix over warps and the tile's count, published
    uint32_t count = 0;
    for (int w = 0; w < SORT_WARPS; ++w) {
        const uint32_t c = sm.wcnt[w][tid];
        sm.wcnt[w][tid] = count;
        count += c;
    }
    uint32_t* mine = status + (size_t)tile * RADIX + tid;
    atomicExch(mine, (tile == 0 ? LB_PREFIX : LB_AGGREGATE) | count);
    // the tile in digit order in shared memory: digit d starts at lstart(d)
    const uint32_t lstart = digit_scan_excl(count, sm.wsum);
    sm.base_d[tid] = lstart;
    __syncthreads();
#pragma unroll
    for (int it = 0; it < ITEMS; ++it) {
        if (wbase + it * 32 + lane < n) {
            const uint32_t d = (kr[it] >> shift) & (RADIX - 1);
            const uint32_t e = sm.base_d[d] + sm.wcnt[warp][d] + rank[it];
            sm.sk[e] = kr[it];
            sm.sv[e] = vr[it];
        }
    }
    uint32_t excl = 0;
    int ok = 1;
    if (tile > 0) {
        // decoupled look-back, LB_BATCH predecessors read at once (independent loads):
        // counts are added from tile - 1 downwards until a tile that holds its inclusive
        // prefix; an unpublished tile is waited for (bounded) and read again
        const unsigned long long t0 = sort_clock_ns();
        int p = tile - 1;
        bool done = false;
        while (!done) {
            uint32_t v[LB_BATCH];
#pragma unroll
            for (int b = 0; b < LB_BATCH; ++b)
                v[b] = p - b >= 0 ? *(volatile uint32_t*)(status + (size_t)(p - b) * RADIX + tid)
                                  : (LB_PREFIX | 0u);
            int b = 0;
            for (; b < LB_BATCH; ++b) {
                if ((v[b] & ~LB_COUNT) == 0u) break;  // not published yet
                excl += v[b] & LB_COUNT;
                if (v[b] & LB_PREFIX) {
                    done = true;
                    break;
                }
            }
            if (done) break;
            p -= b;
            if (b < LB_BATCH) {  // tile p is not published: wait, then read again from it
                if ((*(volatile unsigned*)ctl_status & ST_TIMEOUT) || sort_clock_ns() - t0 > wait_ns) {
                    atomicOr(ctl_status, ST_TIMEOUT);
                    ok = 0;
                    break;
                }
                __nanosleep(32);
            }
        }
        if (ok) atomicExch(mine, LB_PREFIX | (excl + count));
    }
    // global position of the tile's element e of digit d: gbase(d) + excl(d) + e - lstart(d)
    // with gbase the exclusive scan of the pass histogram (the barrier inside the scan
    // also ends every thread's reads of base_d above)
    const uint32_t gstart = digit_scan_excl(ghist[tid], sm.wsum) + excl;
    sm.base_d[tid] = gstart - lstart;  // modulo 2^32: e >= lstart(d) for every element
    if (!__syncthreads_and(ok)) return;
    const int valid_n = min(TILE, n - tile * TILE);
    for (int e = tid; e < valid_n; e += SORT_THREADS) {
        const uint32_t key = sm.sk[e];
        const uint32_t pos = sm.base_d[(key >> shift) & (RADIX - 1)] + (uint32_t)e;
        if (pos < (uint32_t)n) {
            keys_out[pos] = key;
            vals_out[pos] = sm.sv[e];
        }
    }
}

// Adds the digits of `key` for every pass to the block's shared histograms h[pass][digit]
// (warp-aggregated: one shared atomic per distinct digit in the warp).
__device__ __forceinline__ void digit_hist_add(uint32_t key, bool valid, int passes,
                                               uint32_t (*h)[RADIX]) {
    const unsigned lm = lanemask_lt();
    for (int p = 0; p < passes; ++p) {
        const uint32_t d = valid ? ((key >> (8 * p)) & (RADIX - 1)) : (uint32_t)RADIX;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        if (valid && (peers & lm) == 0u) atomicAdd(&h[p][d], (uint32_t)__popc(peers));
    }
}

// The same lower bound found by an exponential search from a guess (the cell's offset
// at the previous build: particles move less than a cell per step, so it is a few places
// off): O(log distance) dependent loads instead of O(log n).
__device__ __forceinline__ uint32_t cell_offset_near(const uint32_t* __restrict__ skeys, int n,
                                                     uint32_t c, uint32_t guess) {
    int lo, hi;  // the answer lies in [lo, hi]
    int g = guess > (uint32_t)n ? n : (int)guess;
    if (g < n && skeys[g] < c) {  // answer > g: gallop right
        int step = 1;
        lo = g + 1;
        hi = g + 1;
        while (hi < n && skeys[hi] < c) {
            lo = hi + 1;
            step <<= 1;
            hi = g + step < n ? g + step : n;
        }
    } else {  // answer <= g: gallop left
        int step = 1;
        hi = g;
        lo = g;
        while (lo > 0 && skeys[lo - 1] >= c) {
            hi = lo - 1;
            step <<= 1;
            lo = g - step > 0 ? g - step : 0;
        }
    }
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (skeys[mid] < c) lo = mid + 1;
        else hi = mid;
    }
    return (uint32_t)lo;
}

// Cell table entry: number of sorted keys < c (lower bound), for c in [0, ncells].
__device__ __forceinline__ uint32_t cell_offset(const uint32_t* __restrict__ skeys, int n, uint32_t c) {
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (skeys[mid] < c) lo = mid + 1;
        else hi = mid;
    }
    return (uint32_t)lo;
}

}  // namespace sph
