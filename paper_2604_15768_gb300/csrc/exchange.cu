// Step 1 and Step 3 of the paper's distributed de-duplication (Sec. 4.1.1,
// Fig. 3) for P virtual ranks on one GPU, as device kernels with no host
// round trip between the steps:
//   rank_join   every entry's key gets its owner rank r in the bits just above
//               the key width, so that ONE sort + unique of the joined keys
//               yields every rank's local sorted distinct run (Step 1), runs in
//               rank order;
//   rank_runs   the rank bits are stripped again and the run boundaries found;
//   exchange    the all-to-all of Step 3: rank q receives, in rank order, the
//               share [bounds[r][q], bounds[r][q+1]) of every run r (the cuts
//               of cusci_partition_plan), gathered into one array with a block
//               per (q, r) segment;
//   split       the final distinct set of the received data (the caller's one
//               dedup over all of it: the ranks' key ranges are disjoint, so
//               the global sort + unique is every rank's final merge at once)
//               is cut at the splitters into the ranks' partitions.

#include "cusci_internal.cuh"

namespace cusci {
namespace {

constexpr int XT = 256;
constexpr int MAX_P = 1024;

int ceil_log2(int P) {
    int b = 0;
    while ((1 << b) < P) b++;
    return b;
}

// bits [lo, lo + nb) of a W-word key set to v (the bits are zero on entry)
template <int W>
__device__ __forceinline__ void put_bits(uint64_t (&k)[W], int lo, int nb, uint64_t v) {
    if (nb == 0) return;
    const int w = lo >> 6, s = lo & 63;
    k[w] |= v << s;
    if (s + nb > 64 && w + 1 < W) k[w + 1] |= v >> (64 - s);
}

template <int W>
__device__ __forceinline__ bool bits_above(const uint64_t (&k)[W], int n_bits) {
    bool any = false;
#pragma unroll
    for (int w = 0; w < W; w++) {
        const int lo = n_bits - 64 * w;  // bits of word w at or above n_bits
        const uint64_t m = lo <= 0 ? ~0ull : (lo >= 64 ? 0ull : (~0ull << lo));
        any |= (k[w] & m) != 0;
    }
    return any;
}

template <int W>
__global__ void __launch_bounds__(XT)
    rank_join(const uint64_t *__restrict__ keys, int64_t total,
              const int64_t *__restrict__ eoff, int P, int n_bits, int lg,
              uint64_t *__restrict__ joint, int32_t *__restrict__ status) {
    __shared__ int64_t eo[MAX_P + 1];
    for (int r = threadIdx.x; r <= P; r += XT) eo[r] = eoff[r];
    __syncthreads();
    for (int64_t e = blockIdx.x * (int64_t)XT + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * XT) {
        uint64_t k[W];
#pragma unroll
        for (int w = 0; w < W; w++) k[w] = keys[e * W + w];
        if (bits_above<W>(k, n_bits) && status) *status = CUSCI_ERR_INVALID;
        // owner rank: the last r with eo[r] <= e
        int lo = 0, hi = P;  // answer in [lo, hi)
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (eo[mid] <= e) lo = mid;
            else hi = mid;
        }
        put_bits<W>(k, n_bits, lg, (uint64_t)lo);
#pragma unroll
        for (int w = 0; w < W; w++) joint[e * W + w] = k[w];
    }
}

// rank of a joined key: bits [n_bits, n_bits + lg)
template <int W>
__device__ __forceinline__ uint32_t rank_of(const uint64_t *k, int n_bits, int lg) {
    if (lg == 0) return 0;
    const int w = n_bits >> 6, s = n_bits & 63;
    uint64_t v = k[w] >> s;
    if (s + lg > 64 && w + 1 < W) v |= k[w + 1] << (64 - s);
    return (uint32_t)(v & ((1ull << lg) - 1ull));
}

template <int W>
__global__ void __launch_bounds__(XT)
    rank_strip(const uint64_t *__restrict__ joint, const int64_t *__restrict__ n_unique,
               int n_bits, uint64_t *__restrict__ runs) {
    const int64_t n = *n_unique;
    for (int64_t i = blockIdx.x * (int64_t)XT + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * XT) {
#pragma unroll
        for (int w = 0; w < W; w++) {
            const int lo = n_bits - 64 * w;
            const uint64_t m = lo <= 0 ? 0ull : (lo >= 64 ? ~0ull : ((1ull << lo) - 1ull));
            runs[i * W + w] = joint[i * W + w] & m;
        }
    }
}

// run_offsets[r] = first position whose rank is >= r (the joined keys are
// sorted by rank first); run_offsets[P] = n_unique
template <int W>
__global__ void rank_bounds(const uint64_t *__restrict__ joint, const int64_t *__restrict__ n_unique,
                            int P, int n_bits, int lg, int64_t *__restrict__ run_off) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r > P) return;
    const int64_t n = *n_unique;
    int64_t lo = 0, hi = n;  // first index in [0, n] with rank >= r
    if (r == P) lo = n;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (rank_of<W>(joint + mid * W, n_bits, lg) < (uint32_t)r) lo = mid + 1;
        else hi = mid;
    }
    run_off[r] = lo;
}

// recv_off[q] = sum over q' < q and all runs r of |share(r, q')|; one block
__global__ void __launch_bounds__(MAX_P)
    recv_sizes(const int64_t *__restrict__ bounds, int P, int64_t *__restrict__ recv_off) {
    __shared__ int64_t sz[MAX_P];
    const int q = threadIdx.x;
    int64_t c = 0;
    if (q < P)
        for (int r = 0; r < P; r++)
            c += bounds[(int64_t)r * (P + 1) + q + 1] - bounds[(int64_t)r * (P + 1) + q];
    sz[q] = q < P ? c : 0;
    __syncthreads();
    if (q == 0) {
        int64_t run = 0;
        for (int i = 0; i < P; i++) {
            recv_off[i] = run;
            run += sz[i];
        }
        recv_off[P] = run;
    }
}

// block (q, r) copies run r's share for rank q to its place in rank q's rows
template <int W>
__global__ void __launch_bounds__(XT)
    exchange_copy(const uint64_t *__restrict__ runs, const int64_t *__restrict__ bounds, int P,
                  const int64_t *__restrict__ recv_off, uint64_t *__restrict__ recv) {
    __shared__ int64_t dst0;
    for (int64_t seg = blockIdx.x; seg < (int64_t)P * P; seg += gridDim.x) {
        const int q = (int)(seg / P), r = (int)(seg % P);
        if (threadIdx.x == 0) {
            int64_t d = recv_off[q];
            for (int rr = 0; rr < r; rr++)
                d += bounds[(int64_t)rr * (P + 1) + q + 1] - bounds[(int64_t)rr * (P + 1) + q];
            dst0 = d;
        }
        __syncthreads();
        const int64_t b0 = bounds[(int64_t)r * (P + 1) + q];
        const int64_t len = bounds[(int64_t)r * (P + 1) + q + 1] - b0;
        const uint64_t *src = runs + b0 * W;
        uint64_t *dst = recv + dst0 * W;
        for (int64_t i = threadIdx.x; i < len * W; i += XT) dst[i] = src[i];
        __syncthreads();  // before dst0 is rewritten
    }
}

template <int W>
__device__ __forceinline__ bool le_w(const uint64_t *a, const uint64_t *b) {
#pragma unroll
    for (int w = W - 1; w >= 0; w--)
        if (a[w] != b[w]) return a[w] < b[w];
    return true;
}

// part_off[q] = number of distinct keys <= splitter[q-1] (q = 1..P-1);
// part_off[0] = 0, part_off[P] = n_unique
template <int W>
__global__ void split_at(const uint64_t *__restrict__ uniq, const int64_t *__restrict__ n_unique,
                         const uint64_t *__restrict__ spl, int P, int64_t *__restrict__ part_off) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q > P) return;
    const int64_t n = *n_unique;
    if (q == 0) { part_off[0] = 0; return; }
    if (q == P) { part_off[P] = n; return; }
    const uint64_t *s = spl + (int64_t)(q - 1) * W;
    int64_t lo = 0, hi = n;  // first index whose key is > s
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (le_w<W>(uniq + mid * W, s)) lo = mid + 1;
        else hi = mid;
    }
    part_off[q] = lo;
}

int grid_for(int64_t n) {
    int64_t g = (n + XT - 1) / XT;
    const int64_t cap = (int64_t)sm_count() * 8;
    if (g > cap) g = cap;
    return (int)(g < 1 ? 1 : g);
}

}  // namespace
}  // namespace cusci

using namespace cusci;

extern "C" cusci_status cusci_rank_join(const uint64_t *d_keys, int W, int64_t total,
                                        const int64_t *d_entry_offsets, int P, int n_bits,
                                        uint64_t *d_joint, int32_t *d_status, void *stream) {
    if ((W != 1 && W != 2) || total < 0 || P < 1 || P > MAX_P || n_bits < 1 ||
        !d_entry_offsets || (total > 0 && (!d_keys || !d_joint)))
        return fail(CUSCI_ERR_INVALID, "cusci_rank_join: bad argument");
    const int lg = ceil_log2(P);
    if (n_bits + lg > 64 * W)
        return fail(CUSCI_ERR_UNSUPPORTED, "cusci_rank_join: %d key bits + %d rank bits exceed %d",
                    n_bits, lg, 64 * W);
    if (total == 0) return CUSCI_OK;
    cudaStream_t st = (cudaStream_t)stream;
    if (W == 1)
        rank_join<1><<<grid_for(total), XT, 0, st>>>(d_keys, total, d_entry_offsets, P, n_bits, lg,
                                                    d_joint, d_status);
    else
        rank_join<2><<<grid_for(total), XT, 0, st>>>(d_keys, total, d_entry_offsets, P, n_bits, lg,
                                                    d_joint, d_status);
    CUSCI_LAUNCHED(1, "rank join");
    return CUSCI_OK;
}

extern "C" cusci_status cusci_rank_runs(const uint64_t *d_joint_unique, int W,
                                        const int64_t *d_n_unique, int64_t capacity, int P,
                                        int n_bits, uint64_t *d_runs, int64_t *d_run_offsets,
                                        void *stream) {
    if ((W != 1 && W != 2) || P < 1 || P > MAX_P || n_bits < 1 || capacity < 0 || !d_n_unique ||
        !d_run_offsets || (capacity > 0 && (!d_joint_unique || !d_runs)))
        return fail(CUSCI_ERR_INVALID, "cusci_rank_runs: bad argument");
    const int lg = ceil_log2(P);
    if (n_bits + lg > 64 * W)
        return fail(CUSCI_ERR_UNSUPPORTED, "cusci_rank_runs: %d key bits + %d rank bits exceed %d",
                    n_bits, lg, 64 * W);
    cudaStream_t st = (cudaStream_t)stream;
    const int gb = (P + 1 + 255) / 256;
    if (W == 1) {
        rank_strip<1><<<grid_for(capacity), XT, 0, st>>>(d_joint_unique, d_n_unique, n_bits, d_runs);
        rank_bounds<1><<<gb, 256, 0, st>>>(d_joint_unique, d_n_unique, P, n_bits, lg, d_run_offsets);
    } else {
        rank_strip<2><<<grid_for(capacity), XT, 0, st>>>(d_joint_unique, d_n_unique, n_bits, d_runs);
        rank_bounds<2><<<gb, 256, 0, st>>>(d_joint_unique, d_n_unique, P, n_bits, lg, d_run_offsets);
    }
    CUSCI_LAUNCHED(2, "rank runs");
    return CUSCI_OK;
}

extern "C" cusci_status cusci_partition_exchange(const uint64_t *d_runs, int W, int P,
                                                 const int64_t *d_bounds, uint64_t *d_recv,
                                                 int64_t *d_recv_offsets, void *stream) {
    if ((W != 1 && W != 2) || P < 1 || P > MAX_P || !d_runs || !d_bounds || !d_recv ||
        !d_recv_offsets)
        return fail(CUSCI_ERR_INVALID, "cusci_partition_exchange: bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    recv_sizes<<<1, MAX_P, 0, st>>>(d_bounds, P, d_recv_offsets);
    int64_t segs = (int64_t)P * P;
    const int64_t cap = (int64_t)sm_count() * 8;
    const int g = (int)(segs < cap ? segs : cap);
    if (W == 1)
        exchange_copy<1><<<g, XT, 0, st>>>(d_runs, d_bounds, P, d_recv_offsets, d_recv);
    else
        exchange_copy<2><<<g, XT, 0, st>>>(d_runs, d_bounds, P, d_recv_offsets, d_recv);
    CUSCI_LAUNCHED(2, "partition exchange");
    return CUSCI_OK;
}

extern "C" cusci_status cusci_partition_split(const uint64_t *d_unique, int W,
                                              const int64_t *d_n_unique,
                                              const uint64_t *d_splitters, int P,
                                              int64_t *d_part_offsets, void *stream) {
    if ((W != 1 && W != 2) || P < 1 || P > MAX_P || !d_unique || !d_n_unique ||
        !d_part_offsets || (P > 1 && !d_splitters))
        return fail(CUSCI_ERR_INVALID, "cusci_partition_split: bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    const int gb = (P + 1 + 255) / 256;
    if (W == 1)
        split_at<1><<<gb, 256, 0, st>>>(d_unique, d_n_unique, d_splitters, P, d_part_offsets);
    else
        split_at<2><<<gb, 256, 0, st>>>(d_unique, d_n_unique, d_splitters, P, d_part_offsets);
    CUSCI_LAUNCHED(1, "partition split");
    return CUSCI_OK;
}
