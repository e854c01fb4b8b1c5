// Streaming two-level top-K selection (Stage 2 of Sec. 3; the running best
// set of Sec. 4.3.4): the K items of largest score seen so far are kept on
// the device; every batch first selects its own K best (local level), which
// are then merged with the running set (global level).  "Best" is exact and
// deterministic: larger score first, equal scores by smaller id.
//
// Selection is an MSD radix select on the 128-bit composite key
// (descending score bits, ascending id): sixteen 8-bit digits, each an
// on-device histogram of the candidates still tied on the higher digits and a
// one-thread pick of the digit holding the K-th key; the items below the
// selected key, plus the key itself, are then compacted.  Scores are
// non-negative FP64 (e.g. |psi| or psi^2); their bit patterns order as their
// values do once -0.0 is read as +0.0.

#include "cusci_internal.cuh"

namespace cusci {
cusci_status exclusive_scan_i64(const int64_t *in, int64_t n, int64_t *out, int64_t *ws,
                                cudaStream_t st);
int64_t scan_tiles(int64_t n);

namespace {

constexpr int KT = 256;

struct SelState {
    unsigned long long prefix_hi, prefix_lo;  // selected digits so far (key bits above the pass)
    long long remaining;                       // rank still to find among the tied candidates
    int bits_done;                             // high bits fixed so far
    int pad;
};

// Composite key of an item: inverted score bits (larger score -> smaller key),
// then the id.  Adding +0.0 first turns -0.0 into +0.0, whose bit pattern is
// the smallest of all non-negative scores (the sign bit of -0.0 would rank it
// above every positive score).
__device__ __forceinline__ void comp_key(double score, int64_t id, uint64_t &hi, uint64_t &lo) {
    hi = ~(uint64_t)__double_as_longlong(__dadd_rn(score, 0.0));
    lo = (uint64_t)id;
}

// digit of the composite key at the 8-bit position `pass` (0 = most significant)
__device__ __forceinline__ uint32_t digit_at(uint64_t hi, uint64_t lo, int pass) {
    return pass < 8 ? (uint32_t)((hi >> (56 - 8 * pass)) & 255)
                    : (uint32_t)((lo >> (56 - 8 * (pass - 8))) & 255);
}

// do the key's bits above the pass equal the selected prefix?
__device__ __forceinline__ bool tied(uint64_t hi, uint64_t lo, const SelState &s) {
    const int b = s.bits_done;
    if (b == 0) return true;
    if (b <= 64) {
        const uint64_t m = b == 64 ? ~0ull : ~(~0ull >> b);
        return (hi & m) == (s.prefix_hi & m);
    }
    const int bl = b - 64;
    const uint64_t m = bl == 64 ? ~0ull : ~(~0ull >> bl);
    return hi == s.prefix_hi && (lo & m) == (s.prefix_lo & m);
}

__global__ void sel_init(SelState *s, long long k, unsigned int *hist) {
    if (threadIdx.x == 0) {
        s->prefix_hi = 0;
        s->prefix_lo = 0;
        s->remaining = k;  // 1-based rank of the key to find
        s->bits_done = 0;
    }
    for (int d = threadIdx.x; d < 256; d += blockDim.x) hist[d] = 0;
}

__global__ void __launch_bounds__(KT)
    sel_hist(const double *__restrict__ sc, const int64_t *__restrict__ id, int64_t n,
             const int64_t *__restrict__ n1p, const double *__restrict__ sc2, const int64_t *__restrict__ id2,
             const int64_t *__restrict__ n2p, const SelState *__restrict__ st, int pass,
             unsigned int *__restrict__ hist, int32_t *__restrict__ status) {
    __shared__ unsigned int h[256];
    for (int d = threadIdx.x; d < 256; d += KT) h[d] = 0;
    __syncthreads();
    const SelState s = *st;
    if (s.bits_done >= 128) return;
    const int64_t n1 = n1p ? *n1p : n;
    const int64_t n2 = n2p ? *n2p : 0;
    const int64_t tot = n1 + n2;
    for (int64_t k = blockIdx.x * (int64_t)KT + threadIdx.x; k < tot;
         k += (int64_t)gridDim.x * KT) {
        uint64_t hi, lo;
        const double v = k < n1 ? sc[k] : sc2[k - n1];
        comp_key(v, k < n1 ? id[k] : id2[k - n1], hi, lo);
        // negative or NaN scores do not order by their bits: reported
        if (pass == 0 && status && !(v >= 0.0)) *status = CUSCI_ERR_INVALID;
        if (tied(hi, lo, s)) atomicAdd(&h[digit_at(hi, lo, pass)], 1u);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < 256; d += KT)
        if (h[d]) atomicAdd(&hist[d], h[d]);
}

// one thread: choose the digit holding the remaining-th key, clear the histogram.
// With fewer candidates than the rank (only possible at the first pass) the
// selected key becomes the largest possible one: every candidate is taken.
__global__ void sel_pick(SelState *st, int pass, unsigned int *hist) {
    if (threadIdx.x == 0) {
        SelState s = *st;
        if (s.bits_done < 128) {
            long long total = 0;
            for (int d = 0; d < 256; d++) total += hist[d];
            if (total < s.remaining) {
                s.prefix_hi = ~0ull;
                s.prefix_lo = ~0ull;
                s.bits_done = 128;
            } else {
                long long acc = 0;
                int d = 0;
                while (acc + (long long)hist[d] < s.remaining) acc += hist[d++];
                s.remaining -= acc;
                if (pass < 8) s.prefix_hi |= (unsigned long long)d << (56 - 8 * pass);
                else s.prefix_lo |= (unsigned long long)d << (56 - 8 * (pass - 8));
                s.bits_done += 8;
                if ((long long)hist[d] == s.remaining) {
                    // every candidate tied on this digit is taken: fill the lower
                    // bits with ones and stop
                    const int b = s.bits_done;
                    if (b < 64) s.prefix_hi |= ~0ull >> b;
                    const int bl = b - 64;
                    if (bl <= 0) s.prefix_lo = ~0ull;
                    else if (bl < 64) s.prefix_lo |= ~0ull >> bl;
                    s.bits_done = 128;
                }
            }
            *st = s;
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 256; i += blockDim.x) hist[i] = 0;
}

// per-tile count of the items with key <= the selected key
__global__ void __launch_bounds__(KT)
    sel_count(const double *__restrict__ sc, const int64_t *__restrict__ id, int64_t n,
              const int64_t *__restrict__ n1p, const double *__restrict__ sc2, const int64_t *__restrict__ id2,
              const int64_t *__restrict__ n2p, const SelState *__restrict__ st,
              int64_t *__restrict__ tile_cnt) {
    const SelState s = *st;
    const int64_t n1 = n1p ? *n1p : n;
    const int64_t n2 = n2p ? *n2p : 0;
    const int64_t k = blockIdx.x * (int64_t)KT + threadIdx.x;
    bool take = false;
    if (k < n1 + n2) {
        uint64_t hi, lo;
        if (k < n1) comp_key(sc[k], id[k], hi, lo);
        else comp_key(sc2[k - n1], id2[k - n1], hi, lo);
        take = hi < s.prefix_hi || (hi == s.prefix_hi && lo <= s.prefix_lo);
    }
    __shared__ int wc[KT / 32];
    const unsigned b = __ballot_sync(0xffffffffu, take);
    if ((threadIdx.x & 31) == 0) wc[threadIdx.x >> 5] = __popc(b);
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t c = 0;
        for (int w = 0; w < KT / 32; w++) c += wc[w];
        tile_cnt[blockIdx.x] = c;
    }
}

__global__ void __launch_bounds__(KT)
    sel_write(const double *__restrict__ sc, const int64_t *__restrict__ id, int64_t n,
              const int64_t *__restrict__ n1p, const double *__restrict__ sc2, const int64_t *__restrict__ id2,
              const int64_t *__restrict__ n2p, const SelState *__restrict__ st,
              const int64_t *__restrict__ tile_off, int64_t cap, double *__restrict__ out_sc,
              int64_t *__restrict__ out_id, int64_t *__restrict__ out_n) {
    const SelState s = *st;
    const int64_t n1 = n1p ? *n1p : n;
    const int64_t n2 = n2p ? *n2p : 0;
    const int64_t k = blockIdx.x * (int64_t)KT + threadIdx.x;
    bool take = false;
    double v = 0.0;
    int64_t ident = 0;
    if (k < n1 + n2) {
        if (k < n1) { v = sc[k]; ident = id[k]; }
        else { v = sc2[k - n1]; ident = id2[k - n1]; }
        uint64_t hi, lo;
        comp_key(v, ident, hi, lo);
        take = hi < s.prefix_hi || (hi == s.prefix_hi && lo <= s.prefix_lo);
    }
    __shared__ int wc[KT / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned b = __ballot_sync(0xffffffffu, take);
    if (lane == 0) wc[wid] = __popc(b);
    __syncthreads();
    int64_t pos = tile_off[blockIdx.x];
    for (int w = 0; w < wid; w++) pos += wc[w];
    pos += __popc(b & ((1u << lane) - 1u));
    if (take && pos < cap) {
        out_sc[pos] = v;
        out_id[pos] = ident;
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) {
        int64_t last = tile_off[blockIdx.x];
        for (int w = 0; w < KT / 32; w++) last += wc[w];
        *out_n = last < cap ? last : cap;
    }
}

size_t al(size_t x) { return (x + 255) & ~(size_t)255; }

// selects the min(K, count) best of (sc, id)[0..n1) and (sc2, id2)[0..n2),
// where n1 / n2 are *n1p / *n2p when given (device counts; n / n2max bound
// them) into (out_sc, out_id), count in *out_n
cusci_status select_best(const double *sc, const int64_t *id, int64_t n, const int64_t *n1p,
                         const double *sc2, const int64_t *id2, const int64_t *n2p, int64_t n2max,
                         int64_t K, double *out_sc, int64_t *out_id, int64_t *out_n,
                         unsigned char *ws, int32_t *status, cudaStream_t st) {
    SelState *state = (SelState *)ws;
    unsigned int *hist = (unsigned int *)(ws + 256);
    const int64_t tot_max = n + n2max;
    const int64_t tiles = (tot_max + KT - 1) / KT;
    int64_t *tile_cnt = (int64_t *)(ws + al(256 + 1024));
    int64_t *tile_off = tile_cnt + al((size_t)(tiles + 1) * 8) / 8;
    int64_t *scan_ws = tile_off + al((size_t)(tiles + 1) * 8) / 8;
    sel_init<<<1, 256, 0, st>>>(state, (long long)K, hist);
    int hb = (int)((tot_max + KT - 1) / KT);
    if (hb > sm_count() * 8) hb = sm_count() * 8;
    if (hb < 1) hb = 1;
    for (int pass = 0; pass < 16; pass++) {
        sel_hist<<<hb, KT, 0, st>>>(sc, id, n, n1p, sc2, id2, n2p, state, pass, hist, status);
        sel_pick<<<1, 256, 0, st>>>(state, pass, hist);
    }
    sel_count<<<(unsigned)tiles, KT, 0, st>>>(sc, id, n, n1p, sc2, id2, n2p, state, tile_cnt);
    cusci_status rc = exclusive_scan_i64(tile_cnt, tiles, tile_off, scan_ws, st);
    if (rc != CUSCI_OK) return rc;
    sel_write<<<(unsigned)tiles, KT, 0, st>>>(sc, id, n, n1p, sc2, id2, n2p, state, tile_off, K,
                                              out_sc, out_id, out_n);
    CUSCI_LAUNCHED(1 + 32 + 2, "top-K select");
    return CUSCI_OK;
}

size_t sel_bytes(int64_t tot) {
    const int64_t tiles = (tot + KT - 1) / KT;
    return al(256 + 1024) + 2 * al((size_t)(tiles + 1) * 8) +
           al((size_t)(scan_tiles(tiles) + 2) * 8);
}

}  // namespace
}  // namespace cusci

using namespace cusci;

extern "C" cusci_status cusci_topk_workspace(int64_t batch, int64_t K, size_t *bytes) {
    if (!bytes || batch < 0 || K < 1)
        return fail(CUSCI_ERR_INVALID, "cusci_topk_workspace: bad argument");
    const int64_t tot = batch > 2 * K ? batch : 2 * K;
    *bytes = sel_bytes(tot) + 4 * al((size_t)K * 8) + al(16);
    return CUSCI_OK;
}

extern "C" cusci_status cusci_topk_update(const double *d_scores, const int64_t *d_ids, int64_t n,
                                          int64_t K, double *d_best_scores, int64_t *d_best_ids,
                                          int64_t *d_best_count, void *d_ws, size_t ws_bytes,
                                          int32_t *d_status, void *stream) {
    if (K < 1 || n < 0 || !d_best_scores || !d_best_ids || !d_best_count ||
        (n > 0 && (!d_scores || !d_ids)))
        return fail(CUSCI_ERR_INVALID, "cusci_topk_update: bad argument");
    size_t need = 0;
    cusci_topk_workspace(n, K, &need);
    if (!d_ws || ws_bytes < need)
        return fail(CUSCI_ERR_OOM, "cusci_topk_update: workspace %zu < %zu", ws_bytes, need);
    if ((uintptr_t)d_ws & 255u)
        return fail(CUSCI_ERR_INVALID, "cusci_topk_update: workspace alignment");
    if (n == 0) return CUSCI_OK;
    cudaStream_t st = (cudaStream_t)stream;
    unsigned char *ws = (unsigned char *)d_ws;
    const size_t sel = sel_bytes(n > 2 * K ? n : 2 * K);
    double *loc_sc = (double *)(ws + sel);
    int64_t *loc_id = (int64_t *)(ws + sel + al((size_t)K * 8));
    double *mrg_sc = (double *)(ws + sel + 2 * al((size_t)K * 8));
    int64_t *mrg_id = (int64_t *)(ws + sel + 3 * al((size_t)K * 8));
    int64_t *cnt = (int64_t *)(ws + sel + 4 * al((size_t)K * 8));  // [0] local, [1] merged
    // level 1: the batch's own best K
    cusci_status rc = select_best(d_scores, d_ids, n, nullptr, nullptr, nullptr, nullptr, 0, K,
                                  loc_sc, loc_id, cnt, ws, d_status, st);
    if (rc != CUSCI_OK) return rc;
    // level 2: merged with the running best set
    rc = select_best(d_best_scores, d_best_ids, K, d_best_count, loc_sc, loc_id, cnt, K, K, mrg_sc,
                     mrg_id, cnt + 1, ws, nullptr, st);
    if (rc != CUSCI_OK) return rc;
    cudaError_t e = cudaMemcpyAsync(d_best_scores, mrg_sc, (size_t)K * 8, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_best_ids, mrg_id, (size_t)K * 8, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_best_count, cnt + 1, 8, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "cusci_topk_update: copy back");
    return CUSCI_OK;
}
