// Regular-sampling partition plan of the paper's distributed de-duplication
// (Sec. 4.1.1, Steps 1 and 2; Fig. 3), for P ranks whose locally sorted,
// distinct key runs lie back to back in one device array.
//   Step 1: every run r contributes S samples at positions floor(k |D_r| / S),
//           k = 0..S-1 (an empty run contributes nothing);
//   Step 2: the samples are sorted and P-1 splitters are taken at equal
//           intervals: splitter j = sample at ((j+1) * count) / P - 1 of the
//           sorted sample (count = number of samples);
//           each run is cut by binary search: rank q receives the keys k with
//           splitter[q-1] < k <= splitter[q] (first and last ranks unbounded).
// The samples are sorted by one block with a bitonic network in shared memory;
// the cuts are one thread per (run, splitter).  Step 3 (the all-to-all and the
// final merge) moves data only and is left to the caller.

#include "cusci_internal.cuh"

namespace cusci {
namespace {

constexpr int PT = 1024;
constexpr int MAX_SAMPLE_WORDS = 16384;  // shared-memory sample buffer (128 KiB)

template <int W>
__device__ __forceinline__ bool less_w(const uint64_t *a, const uint64_t *b) {
#pragma unroll
    for (int w = W - 1; w >= 0; w--)
        if (a[w] != b[w]) return a[w] < b[w];
    return false;
}

template <int W>
__global__ void __launch_bounds__(PT)
    sample_sort_splitters(const uint64_t *__restrict__ keys, const int64_t *__restrict__ off,
                          int P, int S, uint64_t *__restrict__ splitters) {
    extern __shared__ uint64_t smp[];  // [pow2][W]
    __shared__ int count;
    if (threadIdx.x == 0) {
        int c = 0;
        for (int r = 0; r < P; r++)
            if (off[r + 1] > off[r]) c += S;
        count = c;
    }
    __syncthreads();
    int n2 = 1;
    while (n2 < count) n2 <<= 1;
    // gather samples (empty runs skipped, padding with all-ones keys sorts last)
    for (int t = threadIdx.x; t < n2; t += PT) {
        uint64_t v[W];
#pragma unroll
        for (int w = 0; w < W; w++) v[w] = ~0ull;
        if (t < count) {
            int r = 0, seen = 0;
            for (; r < P; r++) {
                if (off[r + 1] > off[r]) {
                    if (t < seen + S) break;
                    seen += S;
                }
            }
            const int k = t - seen;
            const int64_t len = off[r + 1] - off[r];
            const int64_t pos = off[r] + (int64_t)(((unsigned __int128)k * (unsigned __int128)len) / S);
#pragma unroll
            for (int w = 0; w < W; w++) v[w] = keys[pos * W + w];
        }
#pragma unroll
        for (int w = 0; w < W; w++) smp[t * W + w] = v[w];
    }
    __syncthreads();
    // bitonic sort of n2 keys
    for (int size = 2; size <= n2; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = threadIdx.x; t < n2; t += PT) {
                const int partner = t ^ stride;
                if (partner > t) {
                    const bool up = (t & size) == 0;
                    uint64_t *a = smp + t * W, *b = smp + partner * W;
                    const bool swap = up ? less_w<W>(b, a) : less_w<W>(a, b);
                    if (swap) {
#pragma unroll
                        for (int w = 0; w < W; w++) {
                            const uint64_t x = a[w];
                            a[w] = b[w];
                            b[w] = x;
                        }
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int j = threadIdx.x; j < P - 1; j += PT) {
        int64_t at = count > 0 ? ((int64_t)(j + 1) * count) / P - 1 : 0;
        if (at < 0) at = 0;
#pragma unroll
        for (int w = 0; w < W; w++) splitters[j * W + w] = count > 0 ? smp[at * W + w] : ~0ull;
    }
}

// bounds[r][q] for q = 1..P-1: first position of run r whose key exceeds splitter q-1
template <int W>
__global__ void cut_runs(const uint64_t *__restrict__ keys, const int64_t *__restrict__ off,
                         int P, const uint64_t *__restrict__ splitters,
                         int64_t *__restrict__ bounds) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= P * (P + 1)) return;
    const int r = t / (P + 1), q = t % (P + 1);
    int64_t b;
    if (q == 0) {
        b = off[r];
    } else if (q == P) {
        b = off[r + 1];
    } else {
        const uint64_t *sp = splitters + (int64_t)(q - 1) * W;
        int64_t lo = off[r], hi = off[r + 1];  // first key > splitter
        while (lo < hi) {
            const int64_t mid = lo + (hi - lo) / 2;
            if (!less_w<W>(sp, keys + mid * W)) lo = mid + 1;
            else hi = mid;
        }
        b = lo;
    }
    bounds[t] = b;
}

}  // namespace
}  // namespace cusci

using namespace cusci;

extern "C" cusci_status cusci_partition_plan(const uint64_t *d_keys, int W,
                                             const int64_t *d_run_offsets, int P, int S,
                                             uint64_t *d_splitters, int64_t *d_bounds,
                                             void *stream) {
    if (!d_keys || !d_run_offsets || !d_splitters || !d_bounds || (W != 1 && W != 2) || P < 1 ||
        S < 1)
        return fail(CUSCI_ERR_INVALID, "cusci_partition_plan: bad argument");
    int n2 = 1;
    while (n2 < P * S) n2 <<= 1;
    if ((int64_t)n2 * W > MAX_SAMPLE_WORDS)
        return fail(CUSCI_ERR_UNSUPPORTED,
                    "cusci_partition_plan: P*S*W = %d exceeds %d sample words", P * S * W,
                    MAX_SAMPLE_WORDS);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t smem = (size_t)n2 * W * 8;
    {
        cusci_status rc = allow_smem(W == 1 ? (const void *)sample_sort_splitters<1>
                                            : (const void *)sample_sort_splitters<2>,
                                     MAX_SAMPLE_WORDS * 8, "cusci_partition_plan: smem attribute");
        if (rc != CUSCI_OK) return rc;
    }
    if (P > 1) {
        if (W == 1)
            sample_sort_splitters<1><<<1, PT, smem, st>>>(d_keys, d_run_offsets, P, S, d_splitters);
        else
            sample_sort_splitters<2><<<1, PT, smem, st>>>(d_keys, d_run_offsets, P, S, d_splitters);
    }
    const int cells = P * (P + 1);
    if (W == 1)
        cut_runs<1><<<(cells + 255) / 256, 256, 0, st>>>(d_keys, d_run_offsets, P, d_splitters,
                                                        d_bounds);
    else
        cut_runs<2><<<(cells + 255) / 256, 256, 0, st>>>(d_keys, d_run_offsets, P, d_splitters,
                                                        d_bounds);
    CUSCI_LAUNCHED(P > 1 ? 2 : 1, "partition plan");
    return CUSCI_OK;
}
