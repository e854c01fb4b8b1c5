// Exclusive prefix sum of int64 counts into CSR offsets (the "scan" half of
// count-then-fill; it replaces the global append counter of Algorithm 1).
// Three phases over tiles of 2048 elements: tile sums, one-block scan of the
// tile sums, tile-local scans plus the tile prefix.

#include <mutex>

#include "cusci_internal.cuh"

namespace cusci {
namespace {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

__device__ __forceinline__ int64_t warp_incl_scan(int64_t x, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

// block-wide exclusive scan of one value per thread; returns the block total
__device__ __forceinline__ int64_t block_excl_scan(int64_t x, int64_t &excl) {
    __shared__ int64_t warp_tot[SCAN_THREADS / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int64_t inc = warp_incl_scan(x, lane);
    if (lane == 31) warp_tot[wid] = inc;
    __syncthreads();
    int64_t base = 0, total = 0;
#pragma unroll
    for (int w = 0; w < SCAN_THREADS / 32; w++) {
        int64_t t = warp_tot[w];
        if (w < wid) base += t;
        total += t;
    }
    __syncthreads();
    excl = base + inc - x;
    return total;
}

__global__ void __launch_bounds__(SCAN_THREADS)
    tile_sums(const int64_t *__restrict__ in, int64_t n, int64_t *__restrict__ sums) {
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    int64_t acc = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; k++) {
        int64_t idx = base + k * SCAN_THREADS + threadIdx.x;
        if (idx < n) acc += in[idx];
    }
    int64_t excl;
    int64_t tot = block_excl_scan(acc, excl);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(SCAN_THREADS)
    scan_sums(int64_t *__restrict__ sums, int64_t nt) {
    int64_t carry = 0;
    for (int64_t b = 0; b < nt; b += SCAN_THREADS) {
        int64_t idx = b + threadIdx.x;
        int64_t x = idx < nt ? sums[idx] : 0;
        int64_t excl;
        int64_t tot = block_excl_scan(x, excl);
        if (idx < nt) sums[idx] = carry + excl;
        carry += tot;
    }
    if (threadIdx.x == 0) sums[nt] = carry;
}

__global__ void __launch_bounds__(SCAN_THREADS)
    tile_scan(const int64_t *__restrict__ in, int64_t n, const int64_t *__restrict__ sums,
              int64_t nt, int64_t *__restrict__ out) {
    __shared__ int64_t tile[SCAN_TILE];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; k++) {
        int64_t idx = base + k * SCAN_THREADS + threadIdx.x;
        tile[k * SCAN_THREADS + threadIdx.x] = idx < n ? in[idx] : 0;
    }
    __syncthreads();
    int64_t v[SCAN_ITEMS], acc = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; k++) {
        v[k] = tile[threadIdx.x * SCAN_ITEMS + k];
        acc += v[k];
    }
    int64_t excl;
    block_excl_scan(acc, excl);
    excl += sums[blockIdx.x];
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; k++) {
        tile[threadIdx.x * SCAN_ITEMS + k] = excl;
        excl += v[k];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; k++) {
        int64_t idx = base + k * SCAN_THREADS + threadIdx.x;
        if (idx < n) out[idx] = tile[k * SCAN_THREADS + threadIdx.x];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = sums[nt];
}

}  // namespace

int64_t scan_tiles(int64_t n) { return (n + SCAN_TILE - 1) / SCAN_TILE; }

// scan for library-internal callers; ws holds scan_tiles(n)+1 int64
cusci_status exclusive_scan_i64(const int64_t *in, int64_t n, int64_t *out, int64_t *ws,
                                cudaStream_t st) {
    if (n == 0) {
        cudaError_t e = cudaMemsetAsync(out, 0, sizeof(int64_t), st);
        return e == cudaSuccess ? CUSCI_OK : cuda_fail(e, "scan: memset");
    }
    const int64_t nt = scan_tiles(n);
    tile_sums<<<(unsigned)nt, SCAN_THREADS, 0, st>>>(in, n, ws);
    scan_sums<<<1, SCAN_THREADS, 0, st>>>(ws, nt);
    tile_scan<<<(unsigned)nt, SCAN_THREADS, 0, st>>>(in, n, ws, nt, out);
    CUSCI_LAUNCHED(3, "exclusive scan");
    return CUSCI_OK;
}

}  // namespace cusci

using namespace cusci;

extern "C" cusci_status cusci_scan_workspace(int64_t n, size_t *bytes) {
    if (!bytes || n < 0) return fail(CUSCI_ERR_INVALID, "cusci_scan_workspace: bad argument");
    *bytes = (size_t)(scan_tiles(n) + 1) * sizeof(int64_t);
    return CUSCI_OK;
}

extern "C" cusci_status cusci_exclusive_scan(const int64_t *d_counts, int64_t n,
                                             int64_t *d_offsets, void *d_ws, size_t ws_bytes,
                                             void *stream) {
    if (n < 0 || !d_offsets || (n > 0 && !d_counts))
        return fail(CUSCI_ERR_INVALID, "cusci_exclusive_scan: bad argument");
    size_t need = (size_t)(scan_tiles(n) + 1) * sizeof(int64_t);
    if (n > 0 && (!d_ws || ws_bytes < need))
        return fail(CUSCI_ERR_OOM, "cusci_exclusive_scan: workspace %zu < %zu bytes", ws_bytes,
                    need);
    if (((uintptr_t)d_ws & 7u) || ((uintptr_t)d_offsets & 7u) || ((uintptr_t)d_counts & 7u))
        return fail(CUSCI_ERR_INVALID, "cusci_exclusive_scan: buffers must be 8-byte aligned");
    return exclusive_scan_i64(d_counts, n, d_offsets, (int64_t *)d_ws, (cudaStream_t)stream);
}

// ---------------------------------------------------------------------------
// Exclusive scan without allocation.
//
// The tile sums of the scan above normally live in a caller-provided
// workspace.  Some callers cannot hand one over: code running inside a
// framework that has reserved the device's memory for its own pool, code in a
// latency-critical loop where cudaMalloc's implicit device-wide
// synchronisation would stall other streams, and bindings that can only pass
// the pointers of existing buffers.  For them the scratch lives in the
// fixed-size array below, which every device that loads this library holds
// until the process exits (CUSCI_SCAN_STATIC_TILES + 1 int64, 512 KiB + 8 B).
// In host code `g_scan_static` names a host-side shadow, not device memory, so
// its device address is looked up once per device with cudaGetSymbolAddress.

namespace cusci {
namespace {

constexpr int64_t CUSCI_SCAN_STATIC_TILES = 65536;   // => n <= 65536 * 2048 counts
static __device__ __align__(256) int64_t g_scan_static[CUSCI_SCAN_STATIC_TILES + 1];

constexpr int MAX_DEVICES = 64;
std::mutex g_static_mu;
int64_t *g_static_ptr[MAX_DEVICES] = {nullptr};

cusci_status static_scratch(int64_t **out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cusci_exclusive_scan_static: cudaGetDevice");
    if (dev < 0 || dev >= MAX_DEVICES)
        return fail(CUSCI_ERR_UNSUPPORTED, "cusci_exclusive_scan_static: device %d >= %d", dev,
                    MAX_DEVICES);
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scan_static);
        if (e != cudaSuccess)
            return cuda_fail(e, "cusci_exclusive_scan_static: cudaGetSymbolAddress");
        g_static_ptr[dev] = (int64_t *)p;
    }
    *out = g_static_ptr[dev];
    return CUSCI_OK;
}

}  // namespace
}  // namespace cusci

extern "C" int64_t cusci_scan_static_max(void) {
    return cusci::CUSCI_SCAN_STATIC_TILES * cusci::SCAN_TILE;
}

extern "C" cusci_status cusci_exclusive_scan_static(const int64_t *d_counts, int64_t n,
                                                    int64_t *d_offsets, void *stream) {
    using namespace cusci;
    if (n < 0 || !d_offsets || (n > 0 && !d_counts))
        return fail(CUSCI_ERR_INVALID, "cusci_exclusive_scan_static: bad argument");
    if (n > CUSCI_SCAN_STATIC_TILES * SCAN_TILE)
        return fail(CUSCI_ERR_UNSUPPORTED,
                    "cusci_exclusive_scan_static: n=%lld exceeds the static scratch limit of "
                    "%lld counts; use cusci_exclusive_scan with a workspace",
                    (long long)n, (long long)(CUSCI_SCAN_STATIC_TILES * SCAN_TILE));
    if (((uintptr_t)d_offsets & 7u) || ((uintptr_t)d_counts & 7u))
        return fail(CUSCI_ERR_INVALID, "cusci_exclusive_scan_static: buffers must be 8-byte aligned");
    int64_t *scratch = nullptr;
    cusci_status rc = static_scratch(&scratch);
    if (rc != CUSCI_OK) return rc;
    // every tile sum is written before it is read, so nothing needs clearing
    return exclusive_scan_i64(d_counts, n, d_offsets, scratch, (cudaStream_t)stream);
}
