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

}  // namespace
}  // namespace cusci

using namespace cusci;

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
