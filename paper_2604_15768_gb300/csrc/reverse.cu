// Just-in-time reverse index (Stage 3 of Sec. 3; Sec. 4.3.4): the position of
// every key of a batch of coupled targets in the sorted distinct set, found by
// search on the GPU instead of being stored for the whole coupled set.  A
// shared-memory index of every STEP-th distinct key narrows each search to one
// window of STEP keys, searched in global memory (its top levels stay in L2).

#include "cusci_internal.cuh"

namespace cusci {
namespace {

constexpr int RT2 = 256;
constexpr int LOG_STEP = 16;                 // one index entry per 65536 distinct keys
constexpr int MAX_INDEX_WORDS = 8192;        // 64 KiB of shared memory

template <int W>
__device__ __forceinline__ int cmp_w(const uint64_t *a, const uint64_t *b) {
#pragma unroll
    for (int w = W - 1; w >= 0; w--)
        if (a[w] != b[w]) return a[w] < b[w] ? -1 : 1;
    return 0;
}

template <int W, typename IDX>
__global__ void __launch_bounds__(RT2)
    reverse_kernel(const uint64_t *__restrict__ uniq, int64_t nu, const uint64_t *__restrict__ keys,
                   int64_t n, IDX *__restrict__ inverse, int32_t *__restrict__ status) {
    extern __shared__ uint64_t top[];  // [ntop][W]: uniq[t << LOG_STEP]
    const int64_t ntop = (nu + (1ll << LOG_STEP) - 1) >> LOG_STEP;
    for (int64_t t = threadIdx.x; t < ntop; t += RT2)
#pragma unroll
        for (int w = 0; w < W; w++) top[t * W + w] = uniq[(t << LOG_STEP) * W + w];
    __syncthreads();
    for (int64_t k = blockIdx.x * (int64_t)RT2 + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * RT2) {
        uint64_t x[W];
#pragma unroll
        for (int w = 0; w < W; w++) x[w] = keys[k * W + w];
        // last index entry <= x
        int64_t lo = 0, hi = ntop - 1;
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) >> 1;
            if (cmp_w<W>(top + mid * W, x) <= 0) lo = mid;
            else hi = mid - 1;
        }
        int64_t a = lo << LOG_STEP;
        int64_t b = a + (1ll << LOG_STEP) < nu ? a + (1ll << LOG_STEP) : nu;
        while (a < b) {  // first position >= x in the window
            const int64_t mid = a + ((b - a) >> 1);
            if (cmp_w<W>(uniq + mid * W, x) < 0) a = mid + 1;
            else b = mid;
        }
        const bool found = a < nu && cmp_w<W>(uniq + a * W, x) == 0;
        inverse[k] = found ? (IDX)a : (IDX)-1;
        if (!found && status) *status = CUSCI_ERR_INVALID;
    }
}

template <int W, typename IDX>
cusci_status launch_rev(const uint64_t *uniq, int64_t nu, const uint64_t *keys, int64_t n,
                        void *inverse, int32_t *status, cudaStream_t st) {
    const int64_t ntop = (nu + (1ll << LOG_STEP) - 1) >> LOG_STEP;
    const size_t smem = (size_t)ntop * W * 8;
    {
        cusci_status rc = allow_smem((const void *)reverse_kernel<W, IDX>, MAX_INDEX_WORDS * 8,
                                     "reverse index: smem attribute");
        if (rc != CUSCI_OK) return rc;
    }
    int64_t blocks = (n + RT2 - 1) / RT2;
    if (blocks > sm_count() * 8) blocks = sm_count() * 8;
    if (blocks < 1) blocks = 1;
    reverse_kernel<W, IDX><<<(int)blocks, RT2, smem, st>>>(uniq, nu, keys, n, (IDX *)inverse,
                                                           status);
    CUSCI_LAUNCHED(1, "reverse index");
    return CUSCI_OK;
}

// ---------------------------------------------------------------- hashed form
// An open-addressing table of the distinct set built once (key words, and the
// key's position as int64; -1 marks a free slot), so that every later lookup
// costs about one random access instead of a search of the sorted set.
// Layout in the caller's buffer: [slots][W] keys, then [slots] positions.
constexpr int HXT = 256;

__host__ __device__ inline uint64_t rev_slots(int64_t n_unique) {
    uint64_t c = 1024;
    while (c < (uint64_t)n_unique + (uint64_t)n_unique / 2) c <<= 1;  // load <= 2/3
    return c;
}

template <int W>
__device__ __forceinline__ uint64_t rev_hash(const uint64_t *k, uint64_t mask) {
    uint64_t x = k[0];
    if (W == 2) x ^= (k[W - 1] + 0x632be59bd9b4e019ull) * 0x9e3779b97f4a7c15ull;
    x ^= x >> 31;
    x *= 0xbf58476d1ce4e5b9ull;
    x ^= x >> 29;
    return x & mask;
}

template <int W>
__global__ void __launch_bounds__(HXT)
    rev_build(const uint64_t *__restrict__ uniq, int64_t nu, uint64_t *__restrict__ tkeys,
              unsigned long long *__restrict__ tpos, uint64_t mask, int32_t *__restrict__ status) {
    for (int64_t i = blockIdx.x * (int64_t)HXT + threadIdx.x; i < nu;
         i += (int64_t)gridDim.x * HXT) {
        uint64_t k[W];
#pragma unroll
        for (int w = 0; w < W; w++) k[w] = uniq[i * W + w];
        uint64_t h = rev_hash<W>(k, mask);
        bool placed = false;
        for (uint64_t probe = 0; probe <= mask && !placed; probe++) {
            if (atomicCAS(tpos + h, ~0ull, (unsigned long long)i) == ~0ull) {
#pragma unroll
                for (int w = 0; w < W; w++) tkeys[h * W + w] = k[w];
                placed = true;
            }
            h = (h + 1) & mask;
        }
        if (!placed && status) *status = CUSCI_ERR_OVERFLOW;
    }
}

template <int W, typename IDX>
__global__ void __launch_bounds__(HXT)
    rev_lookup(const uint64_t *__restrict__ tkeys, const long long *__restrict__ tpos,
               uint64_t mask, const uint64_t *__restrict__ keys, int64_t n,
               IDX *__restrict__ inverse, int32_t *__restrict__ status) {
    for (int64_t e = blockIdx.x * (int64_t)HXT + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * HXT) {
        uint64_t k[W];
#pragma unroll
        for (int w = 0; w < W; w++) k[w] = keys[e * W + w];
        uint64_t h = rev_hash<W>(k, mask);
        long long found = -1;
        for (uint64_t probe = 0; probe <= mask; probe++) {
            const long long p = __ldg(tpos + h);
            if (p < 0) break;
            bool eq = true;
#pragma unroll
            for (int w = 0; w < W; w++) eq &= __ldg(tkeys + h * W + w) == k[w];
            if (eq) {
                found = p;
                break;
            }
            h = (h + 1) & mask;
        }
        inverse[e] = (IDX)found;
        if (found < 0 && status) *status = CUSCI_ERR_INVALID;
    }
}

int rev_grid(int64_t n) {
    int64_t b = (n + HXT - 1) / HXT;
    const int64_t cap = (int64_t)sm_count() * 8;
    if (b > cap) b = cap;
    return (int)(b < 1 ? 1 : b);
}

}  // namespace
}  // namespace cusci

using namespace cusci;

extern "C" cusci_status cusci_reverse_table_bytes(int64_t n_unique, int W, size_t *bytes) {
    if (n_unique < 1 || (W != 1 && W != 2) || !bytes)
        return fail(CUSCI_ERR_INVALID, "cusci_reverse_table_bytes: bad argument");
    const uint64_t slots = rev_slots(n_unique);
    *bytes = (size_t)slots * 8 * W + (size_t)slots * 8;
    return CUSCI_OK;
}

extern "C" cusci_status cusci_reverse_table_build(const uint64_t *d_unique, int64_t n_unique,
                                                  int W, void *d_table, size_t table_bytes,
                                                  int32_t *d_status, void *stream) {
    size_t need = 0;
    cusci_status rc = cusci_reverse_table_bytes(n_unique, W, &need);
    if (rc != CUSCI_OK) return rc;
    if (!d_unique || !d_table || table_bytes < need || ((uintptr_t)d_table & 15u))
        return fail(CUSCI_ERR_INVALID, "cusci_reverse_table_build: bad buffer (%zu < %zu bytes?)",
                    table_bytes, need);
    const uint64_t slots = rev_slots(n_unique);
    uint64_t *tkeys = (uint64_t *)d_table;
    unsigned long long *tpos = (unsigned long long *)(tkeys + slots * W);
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(tpos, 0xff, slots * 8, st);
    if (e != cudaSuccess) return cuda_fail(e, "reverse table: clear");
    if (W == 1)
        rev_build<1><<<rev_grid(n_unique), HXT, 0, st>>>(d_unique, n_unique, tkeys, tpos,
                                                         slots - 1, d_status);
    else
        rev_build<2><<<rev_grid(n_unique), HXT, 0, st>>>(d_unique, n_unique, tkeys, tpos,
                                                         slots - 1, d_status);
    CUSCI_LAUNCHED(1, "reverse table build");
    return CUSCI_OK;
}

extern "C" cusci_status cusci_reverse_index_table(const void *d_table, int64_t n_unique, int W,
                                                  const uint64_t *d_keys, int64_t n,
                                                  void *d_inverse, int index_bytes,
                                                  int32_t *d_status, void *stream) {
    if (n < 0 || n_unique < 1 || (W != 1 && W != 2) || !d_table ||
        (n > 0 && (!d_keys || !d_inverse)))
        return fail(CUSCI_ERR_INVALID, "cusci_reverse_index_table: bad argument");
    if (index_bytes != 4 && index_bytes != 8)
        return fail(CUSCI_ERR_INVALID, "cusci_reverse_index_table: index_bytes must be 4 or 8");
    if (index_bytes == 4 && n_unique >= ((int64_t)1 << 31))
        return fail(CUSCI_ERR_INVALID, "cusci_reverse_index_table: int32 ids need n_unique < 2^31");
    if (n == 0) return CUSCI_OK;
    const uint64_t slots = rev_slots(n_unique);
    const uint64_t *tkeys = (const uint64_t *)d_table;
    const long long *tpos = (const long long *)(tkeys + slots * W);
    cudaStream_t st = (cudaStream_t)stream;
    const int g = rev_grid(n);
    if (W == 1) {
        if (index_bytes == 4)
            rev_lookup<1, int32_t><<<g, HXT, 0, st>>>(tkeys, tpos, slots - 1, d_keys, n,
                                                     (int32_t *)d_inverse, d_status);
        else
            rev_lookup<1, int64_t><<<g, HXT, 0, st>>>(tkeys, tpos, slots - 1, d_keys, n,
                                                     (int64_t *)d_inverse, d_status);
    } else {
        if (index_bytes == 4)
            rev_lookup<2, int32_t><<<g, HXT, 0, st>>>(tkeys, tpos, slots - 1, d_keys, n,
                                                     (int32_t *)d_inverse, d_status);
        else
            rev_lookup<2, int64_t><<<g, HXT, 0, st>>>(tkeys, tpos, slots - 1, d_keys, n,
                                                     (int64_t *)d_inverse, d_status);
    }
    CUSCI_LAUNCHED(1, "reverse index (table)");
    return CUSCI_OK;
}

extern "C" cusci_status cusci_reverse_index(const uint64_t *d_unique, int64_t n_unique, int W,
                                            const uint64_t *d_keys, int64_t n, void *d_inverse,
                                            int index_bytes, int32_t *d_status, void *stream) {
    if (n < 0 || n_unique < 1 || (W != 1 && W != 2) || !d_unique || (n > 0 && (!d_keys || !d_inverse)))
        return fail(CUSCI_ERR_INVALID, "cusci_reverse_index: bad argument");
    if (index_bytes != 4 && index_bytes != 8)
        return fail(CUSCI_ERR_INVALID, "cusci_reverse_index: index_bytes must be 4 or 8");
    if (index_bytes == 4 && n_unique >= ((int64_t)1 << 31))
        return fail(CUSCI_ERR_INVALID, "cusci_reverse_index: int32 ids need n_unique < 2^31");
    const int64_t ntop = (n_unique + (1ll << LOG_STEP) - 1) >> LOG_STEP;
    if (ntop * W > MAX_INDEX_WORDS)
        return fail(CUSCI_ERR_UNSUPPORTED, "cusci_reverse_index: more than %lld distinct keys",
                    (long long)((int64_t)(MAX_INDEX_WORDS / W) << LOG_STEP));
    if (n == 0) return CUSCI_OK;
    cudaStream_t st = (cudaStream_t)stream;
    if (W == 1)
        return index_bytes == 4
                   ? launch_rev<1, int32_t>(d_unique, n_unique, d_keys, n, d_inverse, d_status, st)
                   : launch_rev<1, int64_t>(d_unique, n_unique, d_keys, n, d_inverse, d_status, st);
    return index_bytes == 4
               ? launch_rev<2, int32_t>(d_unique, n_unique, d_keys, n, d_inverse, d_status, st)
               : launch_rev<2, int64_t>(d_unique, n_unique, d_keys, n, d_inverse, d_status, st);
}
