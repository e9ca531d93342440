// Allocation-free cell sort: the neighbour-build sort (cell key per position, stable
// LSD radix sort, cell offset table) for callers that cannot allocate device memory.
// Its scratch is one file-scope device array of fixed size; every GPU that loads the
// library holds it until the process exits.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>

#include "sph.h"
#include "sph_device.cuh"
#include "sph_launch.h"
#include "sort_impl.cuh"

namespace {

using namespace sph;

constexpr int64_t MAX_N = SPH_NOALLOC_MAX_PARTICLES;
constexpr size_t align256(size_t b) { return (b + 255) & ~size_t(255); }
// radix histogram words for MAX_N keys, by the sizing rule launch_radix_sort indexes with
// (one count per digit and tile of SORT_TILE keys, then the digit totals)
constexpr size_t HIST_WORDS = radix_hist_words_for(MAX_N);
static_assert(HIST_WORDS == (size_t)RADIX * ((MAX_N + SORT_TILE - 1) / SORT_TILE) + RADIX,
              "scratch histograms sized for the sort's tile");
constexpr size_t OFF_KEYS0 = 0;
constexpr size_t OFF_KEYS1 = OFF_KEYS0 + align256(MAX_N * 4);
constexpr size_t OFF_VALS = OFF_KEYS1 + align256(MAX_N * 4);
constexpr size_t OFF_HIST = OFF_VALS + align256(MAX_N * 4);
constexpr size_t OFF_CTL = OFF_HIST + align256(HIST_WORDS * 4);
constexpr size_t SCRATCH_BYTES = OFF_CTL + align256(sizeof(Control));

// The scratch. In host code this name is only a stand-in for the symbol, never a device
// address: the address comes from cudaGetSymbolAddress, once per device.
static __device__ __align__(256) unsigned char g_cell_sort_scratch[SCRATCH_BYTES];

std::mutex g_setup_lock;
void* g_scratch_ptr[64] = {nullptr};
int g_sms[64] = {0};

// Messages go where sph_last_error(NULL) reads them (this thread's global message).
sph_status fail(sph_status s, const std::string& msg) {
    set_global_error(msg);
    return s;
}

// Cell key of each position: the same binning arithmetic as the stepped path
// (position rounded once to the pair-loop precision, IEEE divide, floor, clamp).
__global__ void k_noalloc_keys(const double* __restrict__ x, const double* __restrict__ y,
                               const double* __restrict__ z, int n, Grid G, int precision,
                               uint32_t* __restrict__ keys) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double* xs[3] = {x, y, z};
        int c[3] = {0, 0, 0};
        int clamped = 0;
        for (int d = 0; d < G.dim; ++d) {
            const double v = xs[d][i];
            const double xm = precision ? (double)__double2float_rn(v) : v;
            c[d] = cell_coord(xm, G.lo[d], G.cs[d], G.nc[d], &clamped);
        }
        keys[i] = (uint32_t)(c[0] + G.nc[0] * (c[1] + G.nc[1] * c[2]));
    }
}

}  // namespace

extern "C" sph_status sph_cell_sort_noalloc(const sph_domain* domain, const double* x,
                                            const double* y, const double* z, int64_t n,
                                            uint32_t* order, uint32_t* cell_offsets,
                                            int64_t offsets_capacity, int64_t* ncells_out,
                                            void* stream) {
    if (!domain || !ncells_out) return fail(SPH_ERR_INVALID, "domain and ncells_out are required");
    const sph_domain& D = *domain;
    if (D.dim != 2 && D.dim != 3) return fail(SPH_ERR_INVALID, "dim must be 2 or 3");
    if (D.kernel != SPH_KERNEL_QUINTIC && D.kernel != SPH_KERNEL_WENDLAND_C2 &&
        D.kernel != SPH_KERNEL_CUBIC_SPLINE)
        return fail(SPH_ERR_INVALID, "unknown kernel");
    if (D.precision != SPH_PREC_FP64 && D.precision != SPH_PREC_FP32)
        return fail(SPH_ERR_INVALID, "unknown precision");
    if (n < 0) return fail(SPH_ERR_INVALID, "n < 0");
    if (n > MAX_N)
        return fail(SPH_ERR_CAPACITY, "n = " + std::to_string(n) + " exceeds the maximum of " +
                                          std::to_string(MAX_N) + " particles of the fixed scratch");
    // grid: the rule of sph_create
    const double kh = (D.kernel == SPH_KERNEL_QUINTIC ? 3.0 : 2.0) * D.h;
    if (!(D.h > 0.0) || !std::isfinite(kh)) return fail(SPH_ERR_INVALID, "h must be > 0");
    const int R = D.dim == 3 ? 2 : 1;
    Grid G{};
    G.dim = D.dim;
    double ncells = 1.0;
    for (int d = 0; d < 3; ++d) {
        if (d < D.dim) {
            const double ext = D.hi[d] - D.lo[d];
            if (!(ext > 0.0)) return fail(SPH_ERR_INVALID, "empty cell box");
            double nd = std::floor(ext / (kh / R * 1.00001));
            if (nd < 1.0) nd = 1.0;
            if (nd > 1e7) return fail(SPH_ERR_INVALID, "too many cells");
            G.nc[d] = (int)nd;
            G.periodic[d] = D.periodic[d] ? 1 : 0;
            if (G.periodic[d] && G.nc[d] < 2 * R + 1)
                return fail(SPH_ERR_INVALID, "a periodic axis needs at least 2R + 1 cells");
            G.cs[d] = ext / (double)G.nc[d];
            G.lo[d] = D.lo[d];
            G.hi[d] = D.hi[d];
            G.L[d] = ext;
        } else {
            G.nc[d] = 1;
            G.cs[d] = 1.0;
            G.L[d] = 1.0;
            G.hi[d] = 1.0;
        }
        ncells *= G.nc[d];
    }
    if (ncells > 2147483000.0) return fail(SPH_ERR_INVALID, "too many cells");
    G.ncells = (int)ncells;
    *ncells_out = G.ncells;
    if (!cell_offsets) return SPH_OK;  // size query only
    if (offsets_capacity < (int64_t)G.ncells + 1)
        return fail(SPH_ERR_CAPACITY, "cell_offsets holds " + std::to_string(offsets_capacity) +
                                          " entries, " + std::to_string(G.ncells + 1) + " needed");
    if (n > 0 && (!x || !y || (D.dim == 3 && !z) || !order))
        return fail(SPH_ERR_INVALID, "x, y, (z) and order are required");

    // one-time set-up per device: the device address of the scratch array
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(SPH_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= 64) return fail(SPH_ERR_INVALID, "device ordinal out of range");
    void* base = nullptr;
    int sms = 0;
    {
        std::lock_guard<std::mutex> lock(g_setup_lock);
        if (g_scratch_ptr[dev]) {
            // a device reset unloads the module and its array: a cached address that the
            // runtime no longer knows as this device's memory is looked up again
            cudaPointerAttributes a{};
            const cudaError_t pe = cudaPointerGetAttributes(&a, g_scratch_ptr[dev]);
            if (pe != cudaSuccess || a.type != cudaMemoryTypeDevice || a.device != dev) {
                cudaGetLastError();  // clear the error the query may have recorded
                g_scratch_ptr[dev] = nullptr;
            }
        }
        if (!g_scratch_ptr[dev]) {
            void* ptr = nullptr;
            e = cudaGetSymbolAddress(&ptr, g_cell_sort_scratch);
            if (e != cudaSuccess || !ptr)
                return fail(SPH_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            int s = 0;
            e = cudaDeviceGetAttribute(&s, cudaDevAttrMultiProcessorCount, dev);
            if (e != cudaSuccess) return fail(SPH_ERR_CUDA, cudaGetErrorString(e));
            g_sms[dev] = s;
            g_scratch_ptr[dev] = ptr;
        }
        base = g_scratch_ptr[dev];
        sms = g_sms[dev];
    }
    cudaStream_t st = (cudaStream_t)stream;
    char* p = (char*)base;
    uint32_t* keys[2] = {(uint32_t*)(p + OFF_KEYS0), (uint32_t*)(p + OFF_KEYS1)};
    uint32_t* hist = (uint32_t*)(p + OFF_HIST);
    Control* ctl = (Control*)(p + OFF_CTL);
    int passes = radix_passes(G.ncells);
    if (passes < 1) passes = 1;
    // the sorted permutation lands in vals[passes & 1]: make that the caller's buffer
    uint32_t* vals[2];
    vals[passes & 1] = order;
    vals[(passes & 1) ^ 1] = (uint32_t*)(p + OFF_VALS);
    // the kernels read the status word of the control block: it must start at zero
    e = cudaMemsetAsync(ctl, 0, sizeof(Control), st);
    if (e != cudaSuccess) return fail(SPH_ERR_CUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
    const int ni = (int)n;
    if (ni > 0) {
        int blocks = (ni + 255) / 256;
        if (blocks > sms * 8) blocks = sms * 8;
        k_noalloc_keys<<<blocks, 256, 0, st>>>(x, y, z, ni, G, D.precision, keys[0]);
        const int b = launch_radix_sort(keys, vals, ni, passes, hist, ctl, st);
        launch_cell_offsets(keys[b], ni, G.ncells, cell_offsets, ctl, st, sms);
    } else {
        launch_cell_offsets(keys[0], 0, G.ncells, cell_offsets, ctl, st, sms);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(SPH_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
    return SPH_OK;
}
