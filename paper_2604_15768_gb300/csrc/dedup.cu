// In-batch de-duplication: sorted distinct keys plus the reverse index
// (Sec. 4.1 "local sort + unique", the reverse index of Sec. 2.2 / Sec. 3).
//
// Like the paper we sort rather than hash (Sec. 4.1.2: dense uint64 keys suit
// radix sort; hashing pays atomicCAS divergence).  GB300-specific choices:
//  * keys of fixed popcount N in n_bits bits are replaced by their rank in the
//    combinatorial number system, sum_k C(c_k, k+1) over the set positions
//    c_0 < c_1 < ...; for fixed popcount that rank orders exactly like the
//    numeric value of the bitstring, and it needs ceil(log2 C(n_bits, N)) bits
//    instead of n_bits (41 instead of 52 bits for 14 electrons in 52 spin
//    orbitals), which removes radix passes;
//  * LSD radix sort, 8-bit digits, of (rank, original index) pairs with
//    reduce-then-scan over a persistent grid: an upsweep histogram per CTA, a
//    scan of the digit-major histogram, then a downsweep in which each CTA walks
//    its contiguous range tile by tile, ranks the tile stably with warp-private
//    counters (__match_any_sync), sorts it locally in shared memory and writes
//    digit runs with coalesced stores;
//  * a final pass marks run heads, scans them into unique ids, scatters the
//    inverse and un-ranks the distinct keys.

#include <string.h>

#include <mutex>

#include "radix.cuh"

namespace cusci {
bool ss_eligible(int64_t N, int W, int n_bits, int n_ones);
size_t ss_workspace(int64_t N, int W, int n_bits, int n_ones);
cusci_status ss_dedup(const uint64_t *keys, int64_t N, int W, int n_bits, int n_ones, void *ws,
                      size_t ws_bytes, uint64_t *unique, void *inverse, int index_bytes,
                      int64_t *d_n_unique, int32_t *status, cudaStream_t st);
cusci_status exclusive_scan_i64(const int64_t *in, int64_t n, int64_t *out, int64_t *ws,
                                cudaStream_t st);
int64_t scan_tiles(int64_t n);

namespace {

using namespace radix;

__device__ uint64_t g_binom[128 * BINOM_K];    // C(m, k), saturated at 2^64 - 1
__device__ ulonglong2 g_binom2[128 * BINOM_K];  // C(m, k) exact in 128 bits (lo, hi)
bool g_binom_ready[64] = {false};

// ------------------------------------------------------------------ key transform
// mode 0: raw low n_bits bits; mode 1: combinatorial rank in 64 bits (KW 1);
// mode 2: combinatorial rank in 128 bits (KW 2)
template <int W, int KW>
__global__ void prepare_keys(const uint64_t *__restrict__ keys, int64_t total, int n_bits,
                             int n_ones, int mode, Key<KW> *__restrict__ out,
                             uint32_t *__restrict__ idx, int32_t *__restrict__ status) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total;
         k += (int64_t)gridDim.x * blockDim.x) {
        uint64_t x[W];
        bool bad = false;
        int ones = 0;
#pragma unroll
        for (int w = 0; w < W; w++) {
            x[w] = keys[k * W + w];
            int hi = n_bits - 64 * w;
            uint64_t keep = hi >= 64 ? ~0ull : (hi <= 0 ? 0ull : ((1ull << hi) - 1));
            if (x[w] & ~keep) bad = true;
            x[w] &= keep;
            ones += __popcll(x[w]);
        }
        Key<KW> r;
        if (mode == 2) {
            // rank in 128 bits (KW == 2): keys whose rank space exceeds 2^64
            if (ones != n_ones) bad = true;
            uint64_t lo = 0, hi = 0;
            int c = 0;
#pragma unroll
            for (int w = 0; w < W; w++)
                for (uint64_t b = x[w]; b; b &= b - 1) {
                    int pos = 64 * w + __ffsll((long long)b) - 1;
                    c++;
                    if (c < BINOM_K) {
                        const ulonglong2 v = g_binom2[pos * BINOM_K + c];
                        lo += v.x;
                        hi += v.y + (lo < v.x ? 1ull : 0ull);
                    }
                }
            r.w[0] = lo;
            r.w[KW - 1] = hi;
        } else if (mode == 1) {
            if (ones != n_ones) bad = true;
            uint64_t rank = 0;
            int c = 0;
#pragma unroll
            for (int w = 0; w < W; w++)
                for (uint64_t b = x[w]; b; b &= b - 1) {
                    int pos = 64 * w + __ffsll((long long)b) - 1;
                    c++;
                    if (c < BINOM_K) rank += g_binom[pos * BINOM_K + c];
                }
            r.w[0] = rank;
#pragma unroll
            for (int q = 1; q < KW; q++) r.w[q] = 0;
        } else {
#pragma unroll
            for (int q = 0; q < KW; q++) r.w[q] = q < W ? x[q] : 0;
        }
        if (bad && status) *status = CUSCI_ERR_INVALID;
        out[k] = r;
        idx[k] = (uint32_t)k;
    }
}

// ------------------------------------------------------------------ unique + inverse
constexpr int UT = 256, UI = 8, UTILE = UT * UI;

template <int KW>
__global__ void __launch_bounds__(UT)
    head_counts(const Key<KW> *__restrict__ keys, int64_t total, int64_t *__restrict__ cnt) {
    const int64_t base = (int64_t)blockIdx.x * UTILE;
    uint32_t c = 0;
    for (int r = 0; r < UI; r++) {
        int64_t k = base + r * UT + threadIdx.x;
        if (k < total && (k == 0 || !key_eq<KW>(keys[k], keys[k - 1]))) c++;
    }
    __shared__ uint32_t red[UT / 32];
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(FULL, c, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t s = 0;
        for (int w = 0; w < UT / 32; w++) s += red[w];
        cnt[blockIdx.x] = s;
    }
}

// the distinct keys are copied from the input through the index payload (no
// un-ranking)
template <int KW, int W>
__global__ void __launch_bounds__(UT)
    unique_scatter(const Key<KW> *__restrict__ keys, const uint32_t *__restrict__ idx,
                   int64_t total, const int64_t *__restrict__ tile_off, int n_bits,
                   const uint64_t *__restrict__ orig, uint64_t *__restrict__ unique,
                   void *__restrict__ inverse, int index_bytes,
                   int64_t *__restrict__ n_unique) {
    __shared__ uint32_t warp_tot[UT / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t base = (int64_t)blockIdx.x * UTILE;
    // blocked: thread t handles elements base + t*UI .. +UI-1
    uint32_t head[UI], c = 0;
#pragma unroll
    for (int r = 0; r < UI; r++) {
        int64_t k = base + threadIdx.x * UI + r;
        head[r] = (k < total && (k == 0 || !key_eq<KW>(keys[k], keys[k - 1]))) ? 1u : 0u;
        c += head[r];
    }
    uint32_t inc = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(FULL, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) warp_tot[wid] = inc;
    __syncthreads();
    uint32_t wbase = 0;
    for (int w = 0; w < wid; w++) wbase += warp_tot[w];
    int64_t uid = tile_off[blockIdx.x] + wbase + (inc - c) - 1;  // id of the run before
#pragma unroll
    for (int r = 0; r < UI; r++) {
        int64_t k = base + threadIdx.x * UI + r;
        if (k >= total) break;
        uid += head[r];
        const uint32_t oi = idx[k];
        if (index_bytes == 4) reinterpret_cast<int32_t *>(inverse)[oi] = (int32_t)uid;
        else reinterpret_cast<int64_t *>(inverse)[oi] = uid;
        if (head[r]) {
#pragma unroll
            for (int w = 0; w < W; w++) {
                uint64_t x = orig[(int64_t)oi * W + w];
                const int hi = n_bits - 64 * w;
                x &= hi >= 64 ? ~0ull : (hi <= 0 ? 0ull : ((1ull << hi) - 1));
                unique[uid * W + w] = x;
            }
        }
        if (k == total - 1) *n_unique = uid + 1;
    }
}

// ------------------------------------------------------------------ planning
struct Plan {
    int KW, mode, key_bits, passes, grid;
    int64_t per_cta;
    size_t off_k0, off_k1, off_i0, off_i1, off_hist, off_base, off_scanws, off_tiles, off_tileoff,
        bytes;
};

static unsigned __int128 binom128(int m, int k) {
    if (k < 0 || k > m) return 0;
    unsigned __int128 r = 1;
    for (int i = 1; i <= k; i++) {
        r = r * (unsigned)(m - k + i) / (unsigned)i;
        if (r > ((unsigned __int128)1 << 100)) return (unsigned __int128)1 << 100;
    }
    return r;
}

static int bitlen128(unsigned __int128 x) {
    int b = 0;
    while (x) { b++; x >>= 1; }
    return b;
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

static Plan make_plan(int64_t total, int W, int n_bits, int n_ones) {
    Plan p;
    memset(&p, 0, sizeof(p));
    const unsigned __int128 space = n_ones >= 0 ? binom128(n_bits, n_ones) : 0;
    const unsigned __int128 two64 = (unsigned __int128)1 << 64;
    const unsigned __int128 sat = (unsigned __int128)1 << 100;
    if (n_ones >= 0 && n_ones < BINOM_K && space >= 1 && space <= two64) {
        p.mode = 1;
        p.KW = 1;
        p.key_bits = bitlen128(space - 1);
    } else if (W == 2 && n_ones >= 0 && n_ones < BINOM_K && space > two64 && space < sat &&
               bitlen128(space - 1) < n_bits) {
        p.mode = 2;
        p.KW = 2;
        p.key_bits = bitlen128(space - 1);
    } else {
        p.mode = 0;
        p.KW = n_bits <= 64 ? 1 : W;  // high words of narrow keys are zero
        p.key_bits = n_bits;
    }
    if (p.key_bits < 1) p.key_bits = 1;
    p.passes = (p.key_bits + RBITS - 1) / RBITS;
    int64_t tiles = (total + RTILE - 1) / RTILE;
    // resident blocks per SM of the downsweep (registers bound it: 3 for
    // two-word keys, 4 for one-word keys)
    int64_t g = (int64_t)sm_count() * (p.KW == 2 ? 3 : 4);
    if (g > tiles) g = tiles;
    if (g < 1) g = 1;
    int64_t tiles_per = (tiles + g - 1) / g;
    p.per_cta = tiles_per * RTILE;
    p.grid = (int)((total + p.per_cta - 1) / p.per_cta);
    if (p.grid < 1) p.grid = 1;
    const size_t kb = (size_t)total * 8 * p.KW;
    size_t off = 0;
    p.off_k0 = off; off = align256(off + kb);
    p.off_k1 = off; off = align256(off + kb);
    p.off_i0 = off; off = align256(off + (size_t)total * 4);
    p.off_i1 = off; off = align256(off + (size_t)total * 4);
    const int64_t nh = (int64_t)RADIX * p.grid;
    p.off_hist = off; off = align256(off + (size_t)nh * 4);
    p.off_base = off; off = align256(off + (size_t)(nh + 1) * 8);
    const int64_t ut = (total + UTILE - 1) / UTILE;
    int64_t scan_n = nh > ut ? nh : ut;
    p.off_scanws = off; off = align256(off + (size_t)(scan_tiles(scan_n) + 2) * 8);
    p.off_tiles = off; off = align256(off + (size_t)(ut + 1) * 8);
    p.off_tileoff = off; off = align256(off + (size_t)(ut + 1) * 8);
    p.bytes = off;
    return p;
}

__global__ void widen_hist(const uint32_t *__restrict__ h, int64_t n, int64_t *__restrict__ o) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x)
        o[k] = h[k];
}

cusci_status ensure_binom() {
    static std::mutex mu;
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return fail(CUSCI_ERR_INVALID, "dedup: device id out of range");
    std::lock_guard<std::mutex> lk(mu);
    if (g_binom_ready[dev]) return CUSCI_OK;
    static uint64_t host[128 * BINOM_K];
    static ulonglong2 host2[128 * BINOM_K];
    static unsigned __int128 pas[128][BINOM_K];
    for (int m = 0; m < 128; m++)
        for (int k = 0; k < BINOM_K; k++) {
            unsigned __int128 v;
            if (k == 0) v = 1;
            else if (m == 0) v = 0;
            else v = pas[m - 1][k - 1] + pas[m - 1][k];  // at most C(127, 63) < 2^124
            pas[m][k] = v;
            host[m * BINOM_K + k] = v > (unsigned __int128)(~0ull) ? ~0ull : (uint64_t)v;
            host2[m * BINOM_K + k] = make_ulonglong2((uint64_t)v, (uint64_t)(v >> 64));
        }
    cudaError_t e = cudaMemcpyToSymbol(g_binom, host, sizeof(host));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_binom2, host2, sizeof(host2));
    if (e != cudaSuccess) return cuda_fail(e, "dedup: binomial table upload");
    g_binom_ready[dev] = true;
    return CUSCI_OK;
}

template <int KW, int W>
cusci_status run_dedup(const Plan &p, const uint64_t *d_keys, int64_t total, int n_bits,
                       int n_ones, unsigned char *ws, uint64_t *d_unique, void *d_inverse,
                       int index_bytes, int64_t *d_n_unique, int32_t *d_status, cudaStream_t st) {
    Key<KW> *k0 = (Key<KW> *)(ws + p.off_k0), *k1 = (Key<KW> *)(ws + p.off_k1);
    uint32_t *i0 = (uint32_t *)(ws + p.off_i0), *i1 = (uint32_t *)(ws + p.off_i1);
    uint32_t *hist = (uint32_t *)(ws + p.off_hist);
    int64_t *base = (int64_t *)(ws + p.off_base);
    int64_t *scanws = (int64_t *)(ws + p.off_scanws);
    int64_t *tiles = (int64_t *)(ws + p.off_tiles);
    int64_t *tileoff = (int64_t *)(ws + p.off_tileoff);
    const int ew_blocks = sm_count() * 8;

    prepare_keys<W, KW><<<ew_blocks, 256, 0, st>>>(d_keys, total, n_bits, n_ones, p.mode, k0, i0,
                                                    d_status);
    CUSCI_LAUNCHED(1, "dedup prepare");
    const size_t smem = sizeof(DownSmem<KW>);
    {
        cusci_status rc = allow_smem((const void *)downsweep<KW>, smem, "dedup: smem attribute");
        if (rc != CUSCI_OK) return rc;
    }
    const int64_t nh = (int64_t)RADIX * p.grid;
    for (int pass = 0; pass < p.passes; pass++) {
        const int shift = pass * RBITS;
        upsweep<KW><<<p.grid, RT, 0, st>>>(k0, total, shift, p.per_cta, hist);
        widen_hist<<<64, 256, 0, st>>>(hist, nh, base + 0);
        // in-place exclusive scan: copy counts to the scan input
        cusci_status rc = exclusive_scan_i64(base, nh, base, scanws, st);
        if (rc != CUSCI_OK) return rc;
        downsweep<KW><<<p.grid, RT, smem, st>>>(k0, i0, k1, i1, total, shift, p.per_cta, base);
        CUSCI_LAUNCHED(3, "dedup radix pass");
        Key<KW> *tk = k0; k0 = k1; k1 = tk;
        uint32_t *ti = i0; i0 = i1; i1 = ti;
    }
    const int64_t ut = (total + UTILE - 1) / UTILE;
    head_counts<KW><<<(unsigned)ut, UT, 0, st>>>(k0, total, tiles);
    cusci_status rc = exclusive_scan_i64(tiles, ut, tileoff, scanws, st);
    if (rc != CUSCI_OK) return rc;
    unique_scatter<KW, W><<<(unsigned)ut, UT, 0, st>>>(k0, i0, total, tileoff, n_bits, d_keys,
                                                       d_unique, d_inverse, index_bytes,
                                                       d_n_unique);
    CUSCI_LAUNCHED(2, "dedup unique");
    return CUSCI_OK;
}

}  // namespace
}  // namespace cusci

using namespace cusci;

extern "C" cusci_status cusci_dedup_workspace(int64_t total, int W, int n_bits, int n_ones,
                                              size_t *bytes) {
    if (!bytes || total < 0 || (W != 1 && W != 2) || n_bits < 1 || n_bits > 64 * W)
        return fail(CUSCI_ERR_INVALID, "cusci_dedup_workspace: bad argument");
    if (total >= ((int64_t)1 << 32))
        return fail(CUSCI_ERR_UNSUPPORTED, "cusci_dedup_workspace: total >= 2^32");
    *bytes = ss_eligible(total, W, n_bits, n_ones) ? ss_workspace(total, W, n_bits, n_ones)
                                                   : make_plan(total, W, n_bits, n_ones).bytes;
    return CUSCI_OK;
}

extern "C" cusci_status cusci_dedup(const uint64_t *d_keys, int64_t total, int W, int n_bits,
                                    int n_ones, void *d_ws, size_t ws_bytes, uint64_t *d_unique,
                                    void *d_inverse, int index_bytes, int64_t *d_n_unique,
                                    int64_t *h_n_unique, int32_t *d_status, void *stream) {
    if (total < 0 || (W != 1 && W != 2) || n_bits < 1 || n_bits > 64 * W)
        return fail(CUSCI_ERR_INVALID, "cusci_dedup: bad sizes (total=%lld W=%d n_bits=%d)",
                    (long long)total, W, n_bits);
    if (index_bytes != 4 && index_bytes != 8)
        return fail(CUSCI_ERR_INVALID, "cusci_dedup: index_bytes must be 4 or 8");
    if (!d_n_unique) return fail(CUSCI_ERR_INVALID, "cusci_dedup: d_n_unique is NULL");
    if (total >= ((int64_t)1 << 32))
        return fail(CUSCI_ERR_UNSUPPORTED, "cusci_dedup: total >= 2^32");
    if (index_bytes == 4 && total >= ((int64_t)1 << 31))
        return fail(CUSCI_ERR_INVALID, "cusci_dedup: int32 inverse needs total < 2^31");
    cudaStream_t st = (cudaStream_t)stream;
    if (total == 0) {
        cudaError_t e = cudaMemsetAsync(d_n_unique, 0, sizeof(int64_t), st);
        if (e != cudaSuccess) return cuda_fail(e, "cusci_dedup: memset");
        if (h_n_unique) {
            e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) return cuda_fail(e, "cusci_dedup: sync");
            *h_n_unique = 0;
        }
        return CUSCI_OK;
    }
    if (!d_keys || !d_unique || !d_inverse)
        return fail(CUSCI_ERR_INVALID, "cusci_dedup: NULL buffer");
    if (((uintptr_t)d_ws & 255u) || ((uintptr_t)d_keys & 7u) || ((uintptr_t)d_unique & 7u) ||
        ((uintptr_t)d_inverse & (index_bytes - 1)) || ((uintptr_t)d_n_unique & 7u))
        return fail(CUSCI_ERR_INVALID, "cusci_dedup: misaligned buffer");
    cusci_status rc;
    if (ss_eligible(total, W, n_bits, n_ones)) {
        if (!d_ws) return fail(CUSCI_ERR_OOM, "cusci_dedup: no workspace");
        rc = ss_dedup(d_keys, total, W, n_bits, n_ones, d_ws, ws_bytes, d_unique, d_inverse,
                      index_bytes, d_n_unique, d_status, st);
        if (rc != CUSCI_OK) return rc;
        if (h_n_unique) {
            cudaError_t e = cudaMemcpyAsync(h_n_unique, d_n_unique, sizeof(int64_t),
                                            cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) return cuda_fail(e, "cusci_dedup: n_unique readback");
        }
        return CUSCI_OK;
    }
    Plan p = make_plan(total, W, n_bits, n_ones);
    if (!d_ws || ws_bytes < p.bytes)
        return fail(CUSCI_ERR_OOM, "cusci_dedup: workspace %zu < %zu bytes", ws_bytes, p.bytes);
    rc = ensure_binom();
    if (rc != CUSCI_OK) return rc;
    unsigned char *ws = (unsigned char *)d_ws;
    if (p.KW == 1 && W == 1)
        rc = run_dedup<1, 1>(p, d_keys, total, n_bits, n_ones, ws, d_unique, d_inverse,
                             index_bytes, d_n_unique, d_status, st);
    else if (p.KW == 1 && W == 2)
        rc = run_dedup<1, 2>(p, d_keys, total, n_bits, n_ones, ws, d_unique, d_inverse,
                             index_bytes, d_n_unique, d_status, st);
    else
        rc = run_dedup<2, 2>(p, d_keys, total, n_bits, n_ones, ws, d_unique, d_inverse,
                             index_bytes, d_n_unique, d_status, st);
    if (rc != CUSCI_OK) return rc;
    if (h_n_unique) {
        cudaError_t e =
            cudaMemcpyAsync(h_n_unique, d_n_unique, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, "cusci_dedup: n_unique readback");
    }
    return CUSCI_OK;
}
