// Sample-sort de-duplication: the paper's regular-sampling de-duplication
// (Sec. 4.1.1, Fig. 3) re-thought for one GB300, with the thread blocks of one
// GPU in the role of the paper's ranks.
//
//  1. Regular sampling: OVS samples per leaf bucket are taken at fixed strides
//     of the input, sorted, and every OVS-th sample becomes a splitter
//     (Step 1 and Step 2 of Sec. 4.1.1).  Equal keys always fall into the same
//     bucket; the skewed key distribution (configurations near the reference
//     determinant are far more frequent) is balanced by the sample, not by the
//     key bits.
//  2. Partition in two levels instead of the all-to-all exchange (Step 3): up
//     to a 4096-way split by the level-1 splitters, then a 256-way split of
//     every level-1 bucket, giving leaf buckets of ~1.6k entries (about 1M of
//     them for 1.7e9 keys).  Splitter searches are bracketed by lookup tables
//     over the key range (the sample's range for level 1, the bucket's range
//     for level 2).  The level-1 output is laid out block-major: each block
//     writes its chunk's entries into per-bucket runs inside its own contiguous
//     region, so its write fronts and the later gathers stay inside a few TLB
//     pages and L2 lines.  Slots inside a run are handed out with
//     shared-memory atomics; the slot of every entry is kept
//     (4 B) so the reverse index can be gathered back later.
//  3. Each leaf is de-duplicated in shared memory: every entry is inserted
//     into an open-addressing hash table (its slot kept), the few distinct
//     keys are compacted, packed as (key - leaf_min) << 12 | slot and ordered
//     (rank counting for up to 32 of them; else one counting pass on the top
//     8 bits of their range and counting inside each bucket; 8-bit LSD
//     passes when a bucket is too full), and
//     every entry reads its local unique id back through its slot.  Leaves
//     that are too large or too diverse are LSD-sorted in global memory with
//     their positions in a separate array and walked for run heads.
//  4. A scan of per-leaf distinct counts gives the global unique ids; the
//     distinct keys are compacted, and the reverse index is gathered back
//     through the two stored slot arrays -- reads with the same locality as
//     the scatters, instead of a random 4-byte scatter per entry.
// Keys of at most 64 significant bits are compared as their low word (a second
// word must then be zero); wider two-word keys by their rank in the
// combinatorial number system (order preserving for a fixed number of
// electrons) when it fits 42 bits; other inputs take the LSD path in dedup.cu.

#include <string.h>

#include <mutex>
#include <type_traits>

#include "radix.cuh"

namespace cusci {
cusci_status exclusive_scan_i64(const int64_t *in, int64_t n, int64_t *out, int64_t *ws,
                                cudaStream_t st);
int64_t scan_tiles(int64_t n);

namespace ss {

constexpr int T = 256;
constexpr int WARPS = T / 32;
constexpr int B2 = 256;
constexpr int LOG2_B2 = 8;
using Bid2 = std::conditional<(B2 <= 256), uint8_t, uint16_t>::type;  // leaf id in a bucket
constexpr int OVS = 8;
constexpr int LEAF_AVG = 1600;
constexpr int MAX_B1 = 4096;
constexpr int BT_MAX = 2048;      // binomial-table entries staged in shared memory
constexpr int LRI = 8;            // leaf ranking: entries per thread per tile
constexpr int LTILE = T * LRI;    // 2048
constexpr int MAX_KEY_BITS = 42;   // rank keys: wider ranks sort faster on the LSD path (measured)
constexpr int MAX_RAW_BITS = 64;   // raw single-word keys
constexpr unsigned FULL = 0xffffffffu;
constexpr int LG_CELLS1 = 13;      // level-1 lookup table: 8192 cells over the sampled key range
constexpr int LG_CELLS2 = 10;      // level-2 lookup table per bucket: 1024 cells

struct Plan {
    int64_t N;
    int W, n_bits, n_ones, mode, key_bits, kcols;
    int B1, log2B1;
    int64_t NL, NS;
    int G;
    int64_t per_cta;
    int gs;          // grid of the sample sort
    int64_t gs_per;  // per-CTA range of the sample sort
    int s_passes;
    size_t o_bt, o_samp, o_samp2, o_sidx, o_sidx2, o_shist, o_sbase, o_scanws, o_LS, o_H1,
        o_base1, o_bid1, o_K1, o_dest1, o_bid2, o_K2, o_dest2, o_U2, o_tmpU, o_leafst, o_ucnt,
        o_ubase, o_pay, o_kbase, o_T1, o_krange, bytes;
};

unsigned __int128 binom128(int m, int k) {
    if (k < 0 || k > m) return 0;
    unsigned __int128 r = 1;
    for (int i = 1; i <= k; i++) {
        r = r * (unsigned)(m - k + i) / (unsigned)i;
        if (r > ((unsigned __int128)1 << 100)) return (unsigned __int128)1 << 100;
    }
    return r;
}

int bitlen128(unsigned __int128 x) {
    int b = 0;
    while (x) { b++; x >>= 1; }
    return b;
}

size_t al(size_t x) { return (x + 255) & ~(size_t)255; }

bool eligible(int64_t N, int W, int n_bits, int n_ones, int *mode, int *key_bits) {
    if (N < ((int64_t)1 << 22) || N >= ((int64_t)1 << 32)) return false;
    if (n_bits <= MAX_RAW_BITS) { *mode = 0; *key_bits = n_bits; return true; }
    if (n_ones >= 0 && n_ones < 64 && n_bits * (n_ones + 1) <= BT_MAX) {
        const unsigned __int128 space = binom128(n_bits, n_ones);
        const int kb = space > 1 ? bitlen128(space - 1) : 1;
        if (kb <= MAX_KEY_BITS) { *mode = 1; *key_bits = kb; return true; }
    }
    return false;
}

Plan make_plan(int64_t N, int W, int n_bits, int n_ones, int mode, int key_bits) {
    Plan p;
    memset(&p, 0, sizeof(p));
    p.N = N; p.W = W; p.n_bits = n_bits; p.n_ones = n_ones; p.mode = mode;
    p.key_bits = key_bits;
    p.kcols = mode == 1 ? n_ones + 1 : 1;
    const int64_t want_leaves = (N + LEAF_AVG - 1) / LEAF_AVG;
    int64_t b1 = (want_leaves + B2 - 1) / B2;
    p.B1 = 1; p.log2B1 = 0;
    while (p.B1 < b1 && p.B1 < MAX_B1) { p.B1 <<= 1; p.log2B1++; }
    p.NL = (int64_t)p.B1 * B2;
    p.NS = p.NL * OVS;
    if (p.NS > N) p.NS = N;
    p.G = sm_count() * 3;
    p.per_cta = ((N + p.G - 1) / p.G + 31) / 32 * 32;
    // sample sort grid (radix building blocks)
    const int64_t tiles = (p.NS + radix::RTILE - 1) / radix::RTILE;
    int64_t gs = sm_count() * 4;
    if (gs > tiles) gs = tiles;
    if (gs < 1) gs = 1;
    const int64_t tpc = (tiles + gs - 1) / gs;
    p.gs_per = tpc * radix::RTILE;
    p.gs = (int)((p.NS + p.gs_per - 1) / p.gs_per);
    p.s_passes = (key_bits + radix::RBITS - 1) / radix::RBITS;
    size_t o = 0;
    p.o_bt = o; o = al(o + BT_MAX * 8);
    p.o_samp = o; o = al(o + p.NS * 8);
    p.o_samp2 = o; o = al(o + p.NS * 8);
    p.o_sidx = o; o = al(o + p.NS * 4);
    p.o_sidx2 = o; o = al(o + p.NS * 4);
    p.o_shist = o; o = al(o + (size_t)radix::RADIX * p.gs * 4);
    p.o_sbase = o; o = al(o + ((size_t)radix::RADIX * p.gs + 1) * 8);
    int64_t scan_n = (int64_t)p.B1 * p.G;
    if (p.NL > scan_n) scan_n = p.NL;
    if ((int64_t)radix::RADIX * p.gs > scan_n) scan_n = (int64_t)radix::RADIX * p.gs;
    p.o_scanws = o; o = al(o + (scan_tiles(scan_n) + 2) * 8);
    p.o_LS = o; o = al(o + p.NL * 8);
    p.o_H1 = o; o = al(o + (size_t)p.B1 * p.G * 4);
    p.o_base1 = o; o = al(o + ((size_t)p.B1 * p.G + 1) * 8);
    p.o_bid1 = o; o = al(o + N * 2);
    p.o_K1 = o; o = al(o + N * 8);
    p.o_dest1 = o; o = al(o + N * 4);
    p.o_bid2 = o; o = al(o + N * sizeof(Bid2));
    p.o_K2 = o; o = al(o + N * 8);
    p.o_dest2 = o; o = al(o + N * 4);
    p.o_U2 = o; o = al(o + N * 4);
    p.o_tmpU = o; o = al(o + N * 8);
    p.o_leafst = o; o = al(o + (p.NL + 1) * 8);
    p.o_ucnt = o; o = al(o + p.NL * 8);
    p.o_ubase = o; o = al(o + (p.NL + 1) * 8);
    p.o_pay = o; o = al(o + N * 8);
    p.o_kbase = o; o = al(o + ((size_t)p.B1 + 1) * 8);
    p.o_T1 = o; o = al(o + ((size_t)(1 << LG_CELLS1) + 1) * 2);
    p.o_krange = o; o = al(o + 16);
    p.bytes = o;
    return p;
}

// ------------------------------------------------------------------ device helpers
__device__ __forceinline__ void stage(uint64_t *dst, const uint64_t *__restrict__ src, int n) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
}

// sort key of one W-word key: combinatorial rank (mode 1) or raw word (mode 0);
// *ones receives the number of set bits among the low n_bits, or -1 if a bit
// at or above n_bits is set.
template <int W>
__device__ __forceinline__ uint64_t sort_key_v(const uint64_t (&k)[W], int mode, int n_bits,
                                               int kcols, const uint64_t *bt, int *ones) {
    uint64_t r = 0;
    int c = 0;
    bool above = false;
#pragma unroll
    for (int w = 0; w < W; w++) {
        uint64_t x = k[w];
        const int hi = n_bits - 64 * w;
        const uint64_t keep = hi >= 64 ? ~0ull : (hi <= 0 ? 0ull : ((1ull << hi) - 1));
        if (x & ~keep) above = true;
        x &= keep;
        if (mode == 0) {
            if (w == 0) r = x;
            c += __popcll(x);
            continue;
        }
        for (; x; x &= x - 1) {
            const int pos = 64 * w + __ffsll((long long)x) - 1;
            c++;
            if (c < kcols) r += bt[pos * kcols + c];
        }
    }
    *ones = above ? -1 : c;  // -1: bits above n_bits (invalid key)
    return r;
}

template <int W>
__device__ __forceinline__ uint64_t sort_key(const uint64_t *__restrict__ k, int mode, int n_bits,
                                             int kcols, const uint64_t *bt, int *ones) {
    uint64_t v[W];
#pragma unroll
    for (int w = 0; w < W; w++) v[w] = __ldg(k + w);
    return sort_key_v<W>(v, mode, n_bits, kcols, bt, ones);
}

// raw words of the keys i0 + u*stride (u < U), zeros past end
template <int W, int U>
__device__ __forceinline__ void load_keys(const uint64_t *__restrict__ keys, int64_t i0,
                                          int64_t stride, int64_t end, uint64_t (&r)[U][W]) {
#pragma unroll
    for (int u = 0; u < U; u++) {
        const int64_t i = i0 + (int64_t)u * stride;
#pragma unroll
        for (int w = 0; w < W; w++) r[u][w] = i < end ? __ldg(keys + i * W + w) : 0ull;
    }
}

template <int W>
__device__ __forceinline__ void unrank_to(uint64_t r, int mode, int n_bits, int n_ones, int kcols,
                                          const uint64_t *bt, uint64_t *__restrict__ out) {
    uint64_t x[W];
#pragma unroll
    for (int w = 0; w < W; w++) x[w] = 0;
    if (mode == 0) {
        x[0] = r;
    } else {
        int c = n_bits - 1;
        for (int t = n_ones; t >= 1; t--) {
            while (c >= t && bt[c * kcols + t] > r) c--;
            if (c >= t) r -= bt[c * kcols + t];
            if (c >= 0) x[(c >> 6) & (W - 1)] |= 1ull << (c & 63);
            c--;
        }
    }
#pragma unroll
    for (int w = 0; w < W; w++) out[w] = x[w];
}

// number of entries of the sorted array S[0 .. 2^lg) that are < x (S[last] >= x)
__device__ __forceinline__ int count_less(const uint64_t *S, int lg, uint64_t x) {
    int b = 0;
    for (int step = (1 << lg) >> 1; step >= 1; step >>= 1)
        if (S[b + step - 1] < x) b += step;
    return b;
}

// number of entries of S that are < x, knowing it lies in [lo, hi]
__device__ __forceinline__ int count_less_in(const uint64_t *S, int lo, int hi, uint64_t x) {
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (S[mid] < x) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// cell of x in a table of 2^lg cells of width 2^shift starting at kmin
__device__ __forceinline__ int cell_of(uint64_t x, uint64_t kmin, int shift, int lg) {
    if (x <= kmin) return 0;
    const uint64_t c = (x - kmin) >> shift;
    return c >= (uint64_t)((1 << lg) - 1) ? (1 << lg) - 1 : (int)c;
}

// table T[c] = number of splitters S[0..n) below the start of cell c, T[2^lg] = n - 1
__device__ __forceinline__ void build_cells(const uint64_t *S, int lgS, int n, uint64_t kmin,
                                            int shift, int lg, uint16_t *T) {
    for (int c = threadIdx.x; c <= (1 << lg); c += blockDim.x) {
        if (c == (1 << lg)) {
            T[c] = (uint16_t)(n - 1);
        } else {
            const uint64_t off = (uint64_t)c << shift;
            const uint64_t start = (off > ~0ull - kmin) ? ~0ull : kmin + off;
            T[c] = (uint16_t)count_less(S, lgS, start);
        }
    }
}

// ------------------------------------------------------------------ kernels
__global__ void build_bt(uint64_t *bt, int n_bits, int kcols) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    for (int m = 0; m < n_bits; m++)
        for (int k = 0; k < kcols; k++) {
            uint64_t v;
            if (k == 0) v = 1;
            else if (m == 0) v = 0;
            else {
                const uint64_t a = bt[(m - 1) * kcols + k - 1], b = bt[(m - 1) * kcols + k];
                v = (a + b < a) ? ~0ull : a + b;
            }
            bt[m * kcols + k] = v;
        }
}

template <int W>
__global__ void __launch_bounds__(T)
    sample_keys(const uint64_t *__restrict__ keys, int64_t N, int64_t NS, int mode, int n_bits,
                int kcols, const uint64_t *__restrict__ bt_g, uint64_t *__restrict__ samp,
                uint32_t *__restrict__ sidx) {
    __shared__ uint64_t bt[BT_MAX];
    stage(bt, bt_g, n_bits * kcols);
    __syncthreads();
    for (int64_t j = blockIdx.x * (int64_t)T + threadIdx.x; j < NS; j += (int64_t)gridDim.x * T) {
        const int64_t pos = (int64_t)(((unsigned __int128)j * (unsigned __int128)N) / NS);
        int ones;
        samp[j] = sort_key<W>(keys + pos * W, mode, n_bits, kcols, bt, &ones);
        sidx[j] = (uint32_t)j;
    }
}

// level-1 lookup table over the sampled key range [sorted[0], sorted[NS-1]]
__global__ void build_T1(const uint64_t *__restrict__ sorted, int64_t NS,
                         const uint64_t *__restrict__ LS, int B1, int log2B1,
                         uint16_t *__restrict__ T1, uint64_t *__restrict__ krange) {
    __shared__ uint64_t S1[MAX_B1];
    for (int b = threadIdx.x; b < B1; b += blockDim.x) S1[b] = LS[(int64_t)b * B2 + B2 - 1];
    __syncthreads();
    const uint64_t kmin = sorted[0], kmax = sorted[NS - 1];
    const uint64_t span = kmax - kmin;
    const int bits = span == 0 ? 0 : 64 - __clzll((long long)span);
    const int shift = bits > LG_CELLS1 ? bits - LG_CELLS1 : 0;
    if (threadIdx.x == 0) {
        krange[0] = kmin;
        krange[1] = (uint64_t)shift;
    }
    build_cells(S1, log2B1, B1, kmin, shift, LG_CELLS1, T1);
}

__global__ void make_splitters(const uint64_t *__restrict__ sorted, int64_t NS, int64_t NL,
                               uint64_t *__restrict__ LS) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < NL;
         j += (int64_t)gridDim.x * blockDim.x) {
        if (j == NL - 1) {
            LS[j] = ~0ull;
        } else {
            int64_t s = (j + 1) * (NS / NL) - 1;
            if (NS / NL == 0) s = (int64_t)(((double)(j + 1) / NL) * NS) - 1;
            if (s < 0) s = 0;
            if (s >= NS) s = NS - 1;
            LS[j] = sorted[s];
        }
    }
}

constexpr int U1 = 8;   // keys per thread in flight in the partition passes
constexpr int U1S = 16; // ... in the one-word level-1 scatter (17.0 -> 15.5 ms; 16 slows the others)
constexpr int UG = 8;   // gathers in flight per thread in the reverse-index passes
constexpr int UG1 = 16; // ... in the last of them (measured: 4.9 -> 4.6 ms)

template <int W>
__global__ void __launch_bounds__(T)
    hist1(const uint64_t *__restrict__ keys, int64_t N, int64_t per_cta, int mode, int n_bits,
          int n_ones, int kcols, const uint64_t *__restrict__ bt_g,
          const uint64_t *__restrict__ LS, int B1, int log2B1, const uint16_t *__restrict__ T1,
          const uint64_t *__restrict__ krange, uint16_t *__restrict__ bid1,
          uint32_t *__restrict__ H1, int32_t *__restrict__ status) {
    extern __shared__ __align__(16) unsigned char sm[];
    uint64_t *S1 = (uint64_t *)sm;
    uint64_t *bt = S1 + B1;
    uint32_t *h = (uint32_t *)(bt + (mode == 1 ? BT_MAX : 0));
    uint16_t *T1s = (uint16_t *)(h + B1);
    for (int b = threadIdx.x; b < B1; b += T) {
        S1[b] = LS[(int64_t)b * B2 + B2 - 1];
        h[b] = 0;
    }
    for (int c = threadIdx.x; c <= (1 << LG_CELLS1); c += T) T1s[c] = T1[c];
    if (mode == 1) stage(bt, bt_g, n_bits * kcols);
    const uint64_t kmin = krange[0];
    const int kshift = (int)krange[1];
    __syncthreads();
    const int64_t beg = (int64_t)blockIdx.x * per_cta;
    int64_t end = beg + per_cta;
    if (end > N) end = N;
    bool bad = false;
    // the next batch of keys is loaded while the current one is searched
    uint64_t rn[U1][W];
    load_keys<W, U1>(keys, beg + threadIdx.x, T, end, rn);
    for (int64_t i0 = beg + threadIdx.x; i0 < end; i0 += (int64_t)T * U1) {
        uint64_t r[U1][W];
#pragma unroll
        for (int u = 0; u < U1; u++)
#pragma unroll
            for (int w = 0; w < W; w++) r[u][w] = rn[u][w];
        load_keys<W, U1>(keys, i0 + (int64_t)T * U1, T, end, rn);
#pragma unroll
        for (int u = 0; u < U1; u++) {
            const int64_t i = i0 + (int64_t)u * T;
            if (i < end) {
                int ones;
                const uint64_t x = sort_key_v<W>(r[u], mode, n_bits, kcols, bt, &ones);
                if ((n_ones >= 0 && ones != n_ones) || ones < 0) bad = true;
                const int c = cell_of(x, kmin, kshift, LG_CELLS1);
                const int b = count_less_in(S1, T1s[c], T1s[c + 1], x);
                bid1[i] = (uint16_t)b;
                atomicAdd(&h[b], 1u);
            }
        }
    }
    if (bad && status) *status = CUSCI_ERR_INVALID;
    __syncthreads();
    for (int b = threadIdx.x; b < B1; b += T) H1[(int64_t)blockIdx.x * B1 + b] = h[b];
}

// bucket totals over all blocks (level-1 order of the leaf array)
__global__ void bucket_totals(const uint32_t *__restrict__ H1, int G, int B1,
                              int64_t *__restrict__ tot) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < B1; b += gridDim.x * blockDim.x) {
        int64_t s = 0;
        for (int c = 0; c < G; c++) s += H1[(int64_t)c * B1 + b];
        tot[b] = s;
    }
}

__global__ void widen_u32(const uint32_t *__restrict__ h, int64_t n, int64_t *__restrict__ o) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x)
        o[k] = h[k];
}

// exclusive scan of a shared-memory array v[0..n), in place; every thread of
// the block takes part
__device__ void block_excl_scan_smem(uint32_t *v, int n, uint32_t *warp_tot) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int per = (n + T - 1) / T;
    const int beg = threadIdx.x * per;
    uint32_t s = 0;
    for (int k = 0; k < per; k++)
        if (beg + k < n) s += v[beg + k];
    uint32_t inc = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(FULL, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) warp_tot[wid] = inc;
    __syncthreads();
    uint32_t base = 0;
    for (int w = 0; w < wid; w++) base += warp_tot[w];
    uint32_t ex = base + inc - s;
    for (int k = 0; k < per; k++)
        if (beg + k < n) {
            const uint32_t c = v[beg + k];
            v[beg + k] = ex;
            ex += c;
        }
    __syncthreads();
}

// Level-1 scatter: block c writes its chunk's entries into per-bucket runs of
// its own region [c*per_cta, ...), slots from plain shared-memory atomics;
// base1[c][b] receives the run starts (the block-major layout needs only the
// block's own histogram).  The next batch of keys and bucket ids is loaded
// while the current one is scattered.
template <int W>
__global__ void __launch_bounds__(T)
    scatter1(const uint64_t *__restrict__ keys, int64_t N, int64_t per_cta, int mode, int n_bits,
             int kcols, const uint64_t *__restrict__ bt_g, const uint16_t *__restrict__ bid1,
             int B1, const uint32_t *__restrict__ H1, int64_t *__restrict__ base1,
             uint64_t *__restrict__ K1, uint32_t *__restrict__ dest1) {
    constexpr int US = W == 1 ? U1S : U1;  // two-word keys: registers
    extern __shared__ __align__(16) unsigned char sm[];
    uint32_t *run = (uint32_t *)sm;
    uint64_t *bt = (uint64_t *)(sm + (size_t)MAX_B1 * 4);
    __shared__ uint32_t warp_tot[WARPS];
    for (int b = threadIdx.x; b < B1; b += T) run[b] = H1[(int64_t)blockIdx.x * B1 + b];
    if (mode == 1) stage(bt, bt_g, n_bits * kcols);
    __syncthreads();
    block_excl_scan_smem(run, B1, warp_tot);
    const int64_t beg = (int64_t)blockIdx.x * per_cta;
    for (int b = threadIdx.x; b < B1; b += T) base1[(int64_t)blockIdx.x * B1 + b] = beg + run[b];
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) base1[(int64_t)gridDim.x * B1] = N;
    int64_t end = beg + per_cta;
    if (end > N) end = N;
    uint64_t rn[US][W];
    uint32_t bn[US];
    load_keys<W, US>(keys, beg + threadIdx.x, T, end, rn);
#pragma unroll
    for (int u = 0; u < US; u++) {
        const int64_t i = beg + threadIdx.x + (int64_t)u * T;
        bn[u] = i < end ? bid1[i] : 0u;
    }
    for (int64_t i0 = beg + threadIdx.x; i0 < end; i0 += (int64_t)T * US) {
        uint64_t r[US][W];
        uint32_t b[US];
#pragma unroll
        for (int u = 0; u < US; u++) {
            b[u] = bn[u];
#pragma unroll
            for (int w = 0; w < W; w++) r[u][w] = rn[u][w];
        }
        const int64_t i1 = i0 + (int64_t)T * US;
        load_keys<W, US>(keys, i1, T, end, rn);
#pragma unroll
        for (int u = 0; u < US; u++) {
            const int64_t i = i1 + (int64_t)u * T;
            bn[u] = i < end ? bid1[i] : 0u;
        }
#pragma unroll
        for (int u = 0; u < US; u++) {
            const int64_t i = i0 + (int64_t)u * T;
            if (i < end) {
                int ones;
                const uint64_t x = sort_key_v<W>(r[u], mode, n_bits, kcols, bt, &ones);
                const uint32_t d = (uint32_t)beg + atomicAdd(&run[b[u]], 1u);
                K1[d] = x;
                dest1[i] = d;
            }
        }
    }
}

// one block per level-1 bucket: B2-way split into leaf buckets.  The bucket's
// entries sit in G segments (one per level-1 block, CTA-major layout); its
// leaves are written contiguously from kbase[b1].
__global__ void __launch_bounds__(T)
    level2(const uint64_t *__restrict__ K1, int64_t N, const int64_t *__restrict__ base1,
           const uint32_t *__restrict__ H1, int G, int B1, const int64_t *__restrict__ kbase,
           const uint64_t *__restrict__ LS, int64_t NL, Bid2 *__restrict__ bid2,
           uint64_t *__restrict__ K2, uint32_t *__restrict__ dest2,
           int64_t *__restrict__ leaf_start) {
    __shared__ uint64_t L[B2];
    __shared__ uint32_t h[B2];
    __shared__ uint32_t run[B2];  // next free slot of every leaf, relative to kbase[b1]
    __shared__ uint16_t T2[(1 << LG_CELLS2) + 1];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int b1 = blockIdx.x;
    const int64_t kb = kbase[b1];
    for (int t = threadIdx.x; t < B2; t += T) {
        L[t] = LS[(int64_t)b1 * B2 + t];
        h[t] = 0;
    }
    // this bucket's keys lie in (S1[b1-1], S1[b1]]: a lookup table over that range
    const uint64_t blo = b1 == 0 ? 0ull : LS[(int64_t)b1 * B2 - 1] + 1;
    const uint64_t bhi = LS[(int64_t)b1 * B2 + B2 - 1];
    const uint64_t bspan = bhi > blo ? bhi - blo : 0ull;
    const int bbits = bspan == 0 ? 0 : 64 - __clzll((long long)bspan);
    const int bshift = bbits > LG_CELLS2 ? bbits - LG_CELLS2 : 0;
    __syncthreads();
    build_cells(L, LOG2_B2, B2, blo, bshift, LG_CELLS2, T2);
    __syncthreads();
    for (int c = wid; c < G; c += WARPS) {
        const int64_t sb = base1[(int64_t)c * B1 + b1];
        const int64_t len = H1[(int64_t)c * B1 + b1];
        for (int64_t k0 = 0; k0 < len; k0 += 32 * U1) {
            uint64_t x[U1];
#pragma unroll
            for (int u = 0; u < U1; u++) {
                const int64_t k = k0 + u * 32 + lane;
                x[u] = k < len ? K1[sb + k] : 0;
            }
#pragma unroll
            for (int u = 0; u < U1; u++) {
                const int64_t k = k0 + u * 32 + lane;
                if (k < len) {
                    const int c = cell_of(x[u], blo, bshift, LG_CELLS2);
                    const int b = count_less_in(L, T2[c], T2[c + 1], x[u]);
                    bid2[sb + k] = (Bid2)b;
                    atomicAdd(&h[b], 1u);
                }
            }
        }
    }
    __syncthreads();
    if (wid == 0) {
        constexpr int PER = B2 / 32;
        uint32_t cnt[PER], sum = 0;
#pragma unroll
        for (int q = 0; q < PER; q++) { cnt[q] = h[lane * PER + q]; sum += cnt[q]; }
        uint32_t inc = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(FULL, inc, o);
            if (lane >= o) inc += y;
        }
        uint32_t ex = inc - sum;
#pragma unroll
        for (int q = 0; q < PER; q++) {
            const int t = lane * PER + q;
            run[t] = ex;
            leaf_start[(int64_t)b1 * B2 + t] = kb + ex;
            ex += cnt[q];
        }
    }
    if (b1 == (int)gridDim.x - 1 && threadIdx.x == 0) leaf_start[NL] = N;
    __syncthreads();
    for (int c = wid; c < G; c += WARPS) {
        const int64_t sb = base1[(int64_t)c * B1 + b1];
        const int64_t len = H1[(int64_t)c * B1 + b1];
        for (int64_t k0 = 0; k0 < len; k0 += 32 * U1) {
            uint64_t x[U1];
            uint32_t bb[U1];
#pragma unroll
            for (int u = 0; u < U1; u++) {
                const int64_t k = k0 + u * 32 + lane;
                bb[u] = (uint32_t)B2;
                x[u] = 0;
                if (k < len) {
                    bb[u] = bid2[sb + k];
                    x[u] = K1[sb + k];
                }
            }
#pragma unroll
            for (int u = 0; u < U1; u++) {
                const int64_t k = k0 + u * 32 + lane;
                if (k < len) {
                    const uint64_t d = (uint64_t)kb + atomicAdd(&run[bb[u]], 1u);
                    K2[d] = x[u];
                    dest2[sb + k] = (uint32_t)d;
                }
            }
        }
    }
}

// Leaf de-duplication.  A leaf of at most HT entries is de-duplicated through
// an open-addressing hash table in shared memory (one probe sequence per entry,
// no sort of the entries themselves): the distinct keys are then compacted,
// packed as (key - leaf_min) << LG_HT | slot and ordered -- by counting ranks
// when there are few of them, else by one counting pass on the top 8 bits of
// their range with counting inside each bucket, or by LSD radix passes when a
// bucket is too full -- and every entry reads its rank back through its slot.
// Leaves with more entries, more than HASH_D distinct keys, a key equal to the
// empty marker or a key range too wide to pack are LSD-sorted in global
// memory with their positions alongside.
constexpr int LG_HT = 12;
constexpr int HT = 1 << LG_HT;     // table slots, and entries of a leaf on the hash path
constexpr int HASH_D = HT / 2;     // distinct keys a leaf may hold on the hash path (load <= 1/2)
constexpr int COUNT_D = 32;        // distinct keys ranked by plain counting
constexpr uint64_t EMPTY = ~0ull;  // marker of a free table slot

struct LsdScratch {
    uint32_t hist[256];
    uint32_t hnext[256];  // histogram of the next pass's digit, built while scattering
    uint32_t run[256];
    uint32_t ttot[256];
    uint16_t wcnt[WARPS][256];
    uint32_t flag;
};

struct LeafSmem {
    uint64_t tab[HT];     // hash table; afterwards the two sort buffers tab and tab + HASH_D
    uint16_t es[HT];      // table slot of every entry of the leaf
    uint16_t dl[HASH_D];  // slots of the distinct keys, in order of first insertion
    union {
        LsdScratch L;
        uint16_t sl[HT];  // rank of the key held in every slot (written after ordering)
    } u;
    uint64_t red_lo[WARPS], red_hi[WARPS];
    uint32_t red_cnt[WARPS];
    uint32_t nd, bad;
};

__device__ __forceinline__ void leaf_hist(const uint64_t *a, int64_t n, int shift, uint32_t *hist) {
    for (int d = threadIdx.x; d < 256; d += T) hist[d] = 0;
    __syncthreads();
    for (int64_t k = threadIdx.x; k < n; k += T) atomicAdd(&hist[(a[k] >> shift) & 255], 1u);
    __syncthreads();
}

// One pass of a stable LSD radix sort of a[0..n) into b[0..n) on the 8-bit
// digit at `shift`; pa / pb: optional 32-bit payload moved along (a, b, pa, pb
// in shared or global memory).  L.hist must hold this digit's histogram; when
// next_shift >= 0 the histogram of the digit at next_shift is built into
// L.hnext while scattering.  Returns false (and moves nothing) when every key
// has the same digit.
template <bool PAYLOAD>
__device__ bool leaf_pass(const uint64_t *a, uint64_t *b, const uint32_t *pa, uint32_t *pb,
                          int64_t n, int shift, int next_shift, LsdScratch &L) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (threadIdx.x == 0) L.flag = 0;
    for (int d = threadIdx.x; d < 256; d += T) L.hnext[d] = 0;
    __syncthreads();
    for (int d = threadIdx.x; d < 256; d += T)
        if (L.hist[d] == (uint32_t)n) L.flag = 1;
    __syncthreads();
    if (L.flag) {
        // nothing moves; the next digit's histogram still has to be built
        if (next_shift >= 0)
            for (int64_t k = threadIdx.x; k < n; k += T)
                atomicAdd(&L.hnext[(a[k] >> next_shift) & 255], 1u);
        __syncthreads();
        return false;
    }
    if (wid == 0) {
        uint32_t c[8], s = 0;
#pragma unroll
        for (int q = 0; q < 8; q++) { c[q] = L.hist[lane * 8 + q]; s += c[q]; }
        uint32_t inc = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(FULL, inc, o);
            if (lane >= o) inc += y;
        }
        uint32_t ex = inc - s;
#pragma unroll
        for (int q = 0; q < 8; q++) { L.run[lane * 8 + q] = ex; ex += c[q]; }
    }
    __syncthreads();
    for (int64_t t0 = 0; t0 < n; t0 += LTILE) {
        for (int q = threadIdx.x; q < WARPS * 256; q += T) (&L.wcnt[0][0])[q] = 0;
        __syncthreads();
        uint64_t v[LRI];
        uint32_t dg[LRI], rk[LRI];
#pragma unroll
        for (int r = 0; r < LRI; r++) {
            const int64_t k = t0 + wid * (LRI * 32) + r * 32 + lane;
            v[r] = k < n ? a[k] : 0;
        }
        const int64_t wbase = t0 + wid * (LRI * 32);
#pragma unroll
        for (int r = 0; r < LRI; r++) {
            const int64_t k = wbase + r * 32 + lane;
            const bool valid = k < n;
            dg[r] = valid ? (uint32_t)((v[r] >> shift) & 255) : 256u;
            rk[r] = 0;
            if (wbase + r * 32 >= n) continue;  // whole round past the end (warp-uniform)
            const unsigned peers = __match_any_sync(FULL, dg[r]);
            const int below = __popc(peers & ((1u << lane) - 1u));
            uint32_t prev = valid ? L.wcnt[wid][dg[r]] : 0;
            rk[r] = prev + below;
            __syncwarp();
            if (valid && below == 0) L.wcnt[wid][dg[r]] = (uint16_t)(prev + __popc(peers));
            __syncwarp();
        }
        __syncthreads();
        for (int d = threadIdx.x; d < 256; d += T) {
            uint32_t s = 0;
#pragma unroll
            for (int w = 0; w < WARPS; w++) {
                const uint32_t c = L.wcnt[w][d];
                L.wcnt[w][d] = (uint16_t)s;
                s += c;
            }
            L.ttot[d] = s;
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < LRI; r++) {
            if (dg[r] < 256) {
                const uint32_t dst = L.run[dg[r]] + L.wcnt[wid][dg[r]] + rk[r];
                b[dst] = v[r];
                if (PAYLOAD) pb[dst] = pa[t0 + wid * (LRI * 32) + r * 32 + lane];
                if (next_shift >= 0) atomicAdd(&L.hnext[(v[r] >> next_shift) & 255], 1u);
            }
        }
        __syncthreads();
        for (int d = threadIdx.x; d < 256; d += T) L.run[d] += L.ttot[d];
        __syncthreads();
    }
    return true;
}

// runs the LSD passes over bits [lo, hi) of a[0..n) (ping-ponging with b);
// returns the buffer holding the sorted keys
template <bool PAYLOAD>
__device__ uint64_t *leaf_sort_bits(uint64_t *a, uint64_t *b, uint32_t *&pa, uint32_t *&pb,
                                    int64_t n, int lo, int hi, LsdScratch &L) {
    if (lo >= hi) return a;
    leaf_hist(a, n, lo, L.hist);
    for (int shift = lo; shift < hi; shift += 8) {
        const int next = shift + 8 < hi ? shift + 8 : -1;
        if (leaf_pass<PAYLOAD>(a, b, pa, pb, n, shift, next, L)) {
            uint64_t *t = a; a = b; b = t;
            if (PAYLOAD) { uint32_t *tp = pa; pa = pb; pb = tp; }
        }
        for (int d = threadIdx.x; d < 256; d += T) L.hist[d] = L.hnext[d];
        __syncthreads();
    }
    return a;
}

// walks the sorted keys a[0..n) (positions in the low pbits, or in pos[] when
// given) and writes the local unique id of every position and the distinct keys
__device__ void leaf_walk(const uint64_t *a, const uint32_t *pos, int64_t n, int pbits,
                          uint64_t r_lo, int64_t ls, uint32_t *__restrict__ U2,
                          uint64_t *__restrict__ tmpU, int64_t *__restrict__ ucnt_out,
                          LeafSmem &S) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t chunk = ((n + WARPS - 1) / WARPS + 31) / 32 * 32;
    const int64_t wb = wid * chunk;
    const int64_t we = wb + chunk < n ? wb + chunk : n;
    const uint64_t pmask = pbits == 0 ? 0ull : (~0ull >> (64 - pbits));
    uint32_t cnt = 0;
    for (int64_t k = wb + lane; k < we + 31 && k - lane < we; k += 32) {
        bool head = false;
        if (k < we) head = (k == 0) || ((a[k - 1] >> pbits) != (a[k] >> pbits));
        cnt += __popc(__ballot_sync(FULL, head));
    }
    if (lane == 0) S.red_cnt[wid] = cnt;
    __syncthreads();
    uint32_t base = 0, total = 0;
    for (int w = 0; w < WARPS; w++) {
        const uint32_t c = S.red_cnt[w];
        if (w < wid) base += c;
        total += c;
    }
    for (int64_t k = wb + lane; k - lane < we; k += 32) {
        bool head = false;
        uint64_t v = 0;
        if (k < we) {
            v = a[k];
            head = (k == 0) || ((a[k - 1] >> pbits) != (v >> pbits));
        }
        const unsigned bal = __ballot_sync(FULL, head);
        if (k < we) {
            const uint32_t uid = base + __popc(bal & ((2u << lane) - 1u)) - 1u;
            const int64_t p = pos ? (int64_t)pos[k] : (int64_t)(v & pmask);
            U2[ls + p] = uid;
            if (head) tmpU[ls + uid] = (v >> pbits) + r_lo;
        }
        base += __popc(bal);
    }
    if (threadIdx.x == 0) *ucnt_out = total;
    __syncthreads();
}

// block-wide minimum and maximum of one value per thread (through S.red_lo/hi)
__device__ __forceinline__ void block_min_max(uint64_t lo, uint64_t hi, LeafSmem &S,
                                              uint64_t &r_lo, uint64_t &r_hi) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const uint64_t y = __shfl_xor_sync(FULL, lo, o), z = __shfl_xor_sync(FULL, hi, o);
        lo = y < lo ? y : lo;
        hi = z > hi ? z : hi;
    }
    if (lane == 0) { S.red_lo[wid] = lo; S.red_hi[wid] = hi; }
    __syncthreads();
    r_lo = S.red_lo[0];
    r_hi = S.red_hi[0];
    for (int w = 1; w < WARPS; w++) {
        r_lo = S.red_lo[w] < r_lo ? S.red_lo[w] : r_lo;
        r_hi = S.red_hi[w] > r_hi ? S.red_hi[w] : r_hi;
    }
}

// a leaf off the hash path: keys (key - min) LSD-sorted in global memory with
// their positions in a separate array, then walked for run heads
__device__ void leaf_global(uint64_t *__restrict__ K2, uint64_t *__restrict__ scratch,
                            uint32_t *__restrict__ pay, int64_t N, int64_t ls, int64_t n,
                            uint32_t *__restrict__ U2, uint64_t *__restrict__ tmpU,
                            int64_t *__restrict__ ucnt_out, LeafSmem &S) {
    uint64_t lo = ~0ull, hi = 0;
    for (int64_t k = threadIdx.x; k < n; k += T) {
        const uint64_t x = K2[ls + k];
        lo = x < lo ? x : lo;
        hi = x > hi ? x : hi;
    }
    uint64_t r_lo, r_hi;
    block_min_max(lo, hi, S, r_lo, r_hi);
    const int rb = r_hi == r_lo ? 0 : 64 - __clzll((long long)(r_hi - r_lo));
    uint64_t *a = K2 + ls, *b = scratch + ls;
    uint32_t *pa = pay + ls, *pb = pay + N + ls;
    for (int64_t k = threadIdx.x; k < n; k += T) {
        a[k] = K2[ls + k] - r_lo;
        pa[k] = (uint32_t)k;
    }
    __syncthreads();
    a = leaf_sort_bits<true>(a, b, pa, pb, n, 0, rb, S.u.L);
    leaf_walk(a, pa, n, 0, r_lo, ls, U2, tmpU, ucnt_out, S);
}

// slot of key x in the table of 2^lg slots, inserting it if absent (linear
// probing; at most 2^lg probes); fresh tells whether this call inserted it.
// Sets S.bad when x is the empty marker or when no slot was found.
__device__ __forceinline__ uint32_t hash_insert_slot(uint64_t x, int lg, LeafSmem &S,
                                                     bool &fresh) {
    fresh = false;
    if (x == EMPTY) {
        S.bad = 1;
        return 0;
    }
    volatile uint64_t *vt = S.tab;
    const uint32_t mask = (1u << lg) - 1u;
    uint32_t s = (uint32_t)((x * 0x9E3779B97F4A7C15ull) >> (64 - lg));
    for (uint32_t i = 0; i <= mask; i++) {
        uint64_t cur = vt[s];
        if (cur == EMPTY) {
            cur = atomicCAS((unsigned long long *)&S.tab[s], (unsigned long long)EMPTY,
                            (unsigned long long)x);
            if (cur == EMPTY) {
                fresh = true;
                return s;
            }
        }
        if (cur == x) return s;
        s = (s + 1) & mask;
    }
    S.bad = 1;
    return 0;
}

constexpr int MSD_MAX = 128; // largest bucket the one-pass ordering ranks by counting

// Orders the d packed distinct keys in S.tab[0..d) by one counting pass on the
// top 8 bits of their range (rb bits above the LG_HT slot bits) into
// S.tab[HASH_D..), then ranks every key inside its bucket by counting; writes
// each slot's rank to S.u.sl and the keys to tmpU[ls + rank].  Returns false,
// having written nothing but its scratch, when a bucket holds more than
// MSD_MAX keys (the caller then radix-sorts).  Every thread of the block calls
// it; it ends with a barrier when it succeeds.
__device__ bool order_by_top_bits(int d, int rb, uint64_t r_lo, int64_t ls,
                                  uint64_t *__restrict__ tmpU, LeafSmem &S) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint64_t *a = S.tab, *b = S.tab + HASH_D;
    uint32_t *cnt = S.u.L.hist, *start = S.u.L.run, *fill = S.u.L.ttot;
    const int sh = LG_HT + (rb > 8 ? rb - 8 : 0);
    for (int i = threadIdx.x; i < 256; i += T) {
        cnt[i] = 0;
        fill[i] = 0;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < d; i += T) atomicAdd(&cnt[(a[i] >> sh) & 255], 1u);
    __syncthreads();
    if (wid == 0) {
        uint32_t c[8], sum = 0, mx = 0;
#pragma unroll
        for (int q = 0; q < 8; q++) {
            c[q] = cnt[lane * 8 + q];
            sum += c[q];
            mx = c[q] > mx ? c[q] : mx;
        }
        uint32_t inc = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(FULL, inc, o);
            if (lane >= o) inc += y;
            const uint32_t z = __shfl_xor_sync(FULL, mx, o);
            mx = z > mx ? z : mx;
        }
        uint32_t ex = inc - sum;
#pragma unroll
        for (int q = 0; q < 8; q++) {
            start[lane * 8 + q] = ex;
            ex += c[q];
        }
        if (lane == 0) S.u.L.flag = mx;
    }
    __syncthreads();
    if (S.u.L.flag > (uint32_t)MSD_MAX) return false;
    for (int i = threadIdx.x; i < d; i += T) {
        const uint64_t m = a[i];
        const uint32_t g = (uint32_t)(m >> sh) & 255u;
        b[start[g] + atomicAdd(&fill[g], 1u)] = m;
    }
    __syncthreads();
    uint32_t *R = reinterpret_cast<uint32_t *>(a);  // ranks, over the consumed input
    for (int j = threadIdx.x; j < d; j += T) {
        const uint64_t m = b[j];
        const uint32_t g = (uint32_t)(m >> sh) & 255u;
        const int s0 = (int)start[g], s1 = s0 + (int)cnt[g];
        uint32_t r = (uint32_t)s0;
        for (int k = s0; k < s1; k++) r += b[k] < m;
        R[j] = r;
    }
    __syncthreads();  // the scratch read above shares memory with sl
    for (int j = threadIdx.x; j < d; j += T) {
        const uint64_t m = b[j];
        const uint32_t r = R[j];
        S.u.sl[m & (HT - 1)] = (uint16_t)r;
        tmpU[ls + r] = (m >> LG_HT) + r_lo;
    }
    return true;
}

constexpr int DPT = HASH_D / T;  // distinct keys per thread in the compaction

// every slot of the table EMPTY, then a barrier
__device__ __forceinline__ void clear_table(LeafSmem &S) {
    for (int s = threadIdx.x; s < HT; s += T) S.tab[s] = EMPTY;
    __syncthreads();
}
constexpr int UI = 4;        // keys in flight per thread in the insertion

__global__ void __launch_bounds__(T, 4)
    leaf_dedup(uint64_t *__restrict__ K2, uint64_t *__restrict__ scratch,
               uint32_t *__restrict__ pay, int64_t N, int64_t NL,
               const int64_t *__restrict__ leaf_start, uint32_t *__restrict__ U2,
               uint64_t *__restrict__ tmpU, int64_t *__restrict__ ucnt) {
    extern __shared__ __align__(16) unsigned char sm[];
    LeafSmem &S = *reinterpret_cast<LeafSmem *>(sm);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    clear_table(S);
    for (int64_t leaf = blockIdx.x; leaf < NL; leaf += gridDim.x) {
        const int64_t ls = leaf_start[leaf];
        const int64_t n = leaf_start[leaf + 1] - ls;
        if (n <= 0) {
            if (threadIdx.x == 0) ucnt[leaf] = 0;
            continue;
        }
        if (n > HT) {
            leaf_global(K2, scratch, pay, N, ls, n, U2, tmpU, ucnt + leaf, S);
            continue;
        }
        // table of 2^lg >= 2n slots (64 at least, HT at most); all HT slots are
        // EMPTY here (cleared before the first leaf and behind every leaf)
        int lg = (n <= 1 ? 0 : 64 - __clzll((long long)(n - 1))) + 1;
        lg = lg < 6 ? 6 : (lg > LG_HT ? LG_HT : lg);
        if (threadIdx.x == 0) {
            S.bad = 0;
            S.nd = 0;
        }
        __syncthreads();
        // 1. insert every entry, remembering its slot; the slots of new keys are
        //    appended to S.dl (one shared atomic per warp and round)
        for (int64_t k0 = 0; k0 < n; k0 += T * UI) {
            uint64_t x[UI];
#pragma unroll
            for (int u = 0; u < UI; u++) {
                const int64_t k = k0 + u * T + threadIdx.x;
                x[u] = k < n ? K2[ls + k] : 0;
            }
#pragma unroll
            for (int u = 0; u < UI; u++) {
                const int64_t k = k0 + u * T + threadIdx.x;
                bool fresh = false;
                uint32_t slot = 0;
                if (k < n) {
                    slot = hash_insert_slot(x[u], lg, S, fresh);
                    S.es[k] = (uint16_t)slot;
                }
                const unsigned bal = __ballot_sync(FULL, fresh);
                if (bal) {
                    const int lead = __ffs(bal) - 1;
                    uint32_t base = 0;
                    if (lane == lead) base = atomicAdd(&S.nd, (uint32_t)__popc(bal));
                    base = __shfl_sync(FULL, base, lead);
                    const uint32_t i = base + __popc(bal & ((1u << lane) - 1u));
                    if (fresh && i < (uint32_t)HASH_D) S.dl[i] = (uint16_t)slot;
                }
            }
        }
        __syncthreads();
        const int d = (int)S.nd;
        if (S.bad || d > HASH_D) {
            leaf_global(K2, scratch, pay, N, ls, n, U2, tmpU, ucnt + leaf, S);
            clear_table(S);
            continue;
        }
        // 2. the distinct keys (all read before the packed keys overwrite the
        //    table front), their range, and the packed keys in tab[0..d)
        uint64_t v[DPT];
        uint32_t sv[DPT];
        uint64_t lo = ~0ull, hi = 0;
#pragma unroll
        for (int j = 0; j < DPT; j++) {
            const int i = j * T + threadIdx.x;
            sv[j] = 0;
            v[j] = 0;
            if (i < d) {
                sv[j] = S.dl[i];
                v[j] = S.tab[sv[j]];
                lo = v[j] < lo ? v[j] : lo;
                hi = v[j] > hi ? v[j] : hi;
            }
        }
        uint64_t r_lo, r_hi;
        block_min_max(lo, hi, S, r_lo, r_hi);
        const int rb = r_hi == r_lo ? 0 : 64 - __clzll((long long)(r_hi - r_lo));
        if (rb + LG_HT > 64) {
            __syncthreads();  // every thread has read the reductions
            leaf_global(K2, scratch, pay, N, ls, n, U2, tmpU, ucnt + leaf, S);
            clear_table(S);
            continue;
        }
#pragma unroll
        for (int j = 0; j < DPT; j++) {
            const int i = j * T + threadIdx.x;
            if (i < d) S.tab[i] = ((v[j] - r_lo) << LG_HT) | sv[j];
        }
        // rank counters of the counting path, behind the packed keys (d <= T)
        uint32_t *rank = reinterpret_cast<uint32_t *>(S.tab + HASH_D);
        if (d <= COUNT_D && threadIdx.x < d) rank[threadIdx.x] = 0;
        __syncthreads();
        // 3. order the d distinct keys; write each slot's rank and the keys
        if (d <= COUNT_D) {
            // key chunk c (32 keys, one per lane) against a share of all d keys:
            // the C = ceil(d/32) chunks split the block's warps between them
            const uint64_t *a = S.tab;
            const int C = (d + 31) >> 5, sh = WARPS / C;
            if (wid < C * sh) {
                const int c = wid / sh, part = wid % sh;
                const int i = c * 32 + lane;
                const uint64_t m = i < d ? a[i] : 0;
                const int j0 = part * d / sh, j1 = (part + 1) * d / sh;
                uint32_t r = 0;
                int j = j0;
                for (; j + 4 <= j1; j += 4) {
                    r += (a[j] < m) + (a[j + 1] < m);
                    r += (a[j + 2] < m) + (a[j + 3] < m);
                }
                for (; j < j1; j++) r += a[j] < m;
                if (i < d) {
                    if (sh == 1) rank[i] = r;
                    else atomicAdd(&rank[i], r);
                }
            }
            __syncthreads();
            if (threadIdx.x < d) {
                const uint64_t m = a[threadIdx.x];
                const uint32_t r = rank[threadIdx.x];
                S.u.sl[m & (HT - 1)] = (uint16_t)r;
                tmpU[ls + r] = (m >> LG_HT) + r_lo;
            }
        } else if (!order_by_top_bits(d, rb, r_lo, ls, tmpU, S)) {
            uint32_t *np = nullptr, *nq = nullptr;
            const uint64_t *a =
                leaf_sort_bits<false>(S.tab, S.tab + HASH_D, np, nq, d, LG_HT, LG_HT + rb, S.u.L);
            // the radix passes end with a barrier: their scratch may now hold sl
            for (int r = threadIdx.x; r < d; r += T) {
                const uint64_t m = a[r];
                S.u.sl[m & (HT - 1)] = (uint16_t)r;
                tmpU[ls + r] = (m >> LG_HT) + r_lo;
            }
        }
        __syncthreads();
        // 4. the local unique id of every entry; behind it the table is made
        //    EMPTY again where this leaf touched it: the occupied slots, the
        //    packed keys / ranks in [0, d) and the second buffer [HASH_D, +d)
        for (int k = threadIdx.x; k < (int)n; k += T) U2[ls + k] = S.u.sl[S.es[k]];
        for (int i = threadIdx.x; i < d; i += T) {
            S.tab[S.dl[i]] = EMPTY;
            S.tab[i] = EMPTY;
            S.tab[HASH_D + i] = EMPTY;
        }
        if (threadIdx.x == 0) ucnt[leaf] = d;
        __syncthreads();  // before the next leaf inserts
    }
}

template <int W>
__global__ void __launch_bounds__(T)
    compact_unique(const uint64_t *__restrict__ tmpU, const int64_t *__restrict__ leaf_start,
                   const int64_t *__restrict__ ucnt, const int64_t *__restrict__ ubase,
                   int64_t NL, int mode, int n_bits, int n_ones, int kcols,
                   const uint64_t *__restrict__ bt_g, uint64_t *__restrict__ unique,
                   int64_t *__restrict__ n_unique) {
    __shared__ uint64_t bt[BT_MAX];
    if (mode == 1) stage(bt, bt_g, n_bits * kcols);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)T + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * T) >> 5;
    for (int64_t leaf = warp; leaf < NL; leaf += nw) {
        const int64_t ls = leaf_start[leaf], c = ucnt[leaf], ub = ubase[leaf];
        for (int64_t k = lane; k < c; k += 32) {
            if (mode == 0) {
                unique[(ub + k) * W] = tmpU[ls + k];
                if (W == 2) unique[(ub + k) * W + 1] = 0;
            } else {
                unrank_to<W>(tmpU[ls + k], mode, n_bits, n_ones, kcols, bt, unique + (ub + k) * W);
            }
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *n_unique = ubase[NL];
}

__global__ void __launch_bounds__(T)
    unscatter2(const int64_t *__restrict__ base1, const uint32_t *__restrict__ H1, int G, int B1,
               const Bid2 *__restrict__ bid2, uint32_t *__restrict__ dest2_u1,
               const uint32_t *__restrict__ U2, const int64_t *__restrict__ ubase) {
    const int b1 = blockIdx.x;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int c = wid; c < G; c += WARPS) {
        const int64_t sb = base1[(int64_t)c * B1 + b1];
        const int64_t len = H1[(int64_t)c * B1 + b1];
        for (int64_t k0 = 0; k0 < len; k0 += 32 * UG) {
            uint32_t d[UG], lf[UG], u[UG];
#pragma unroll
            for (int q = 0; q < UG; q++) {
                const int64_t k = k0 + q * 32 + lane;
                d[q] = k < len ? dest2_u1[sb + k] : 0u;
                lf[q] = k < len ? bid2[sb + k] : 0u;
            }
#pragma unroll
            for (int q = 0; q < UG; q++) {
                const int64_t k = k0 + q * 32 + lane;
                u[q] = k < len ? U2[d[q]] : 0u;
            }
#pragma unroll
            for (int q = 0; q < UG; q++) {
                const int64_t k = k0 + q * 32 + lane;
                if (k < len)
                    dest2_u1[sb + k] = (uint32_t)(u[q] + ubase[(int64_t)b1 * B2 + lf[q]]);
            }
        }
    }
}

template <typename IDX>
__global__ void __launch_bounds__(256)
    unscatter1(const uint32_t *__restrict__ dest1, const uint32_t *__restrict__ U1v, int64_t N,
               IDX *__restrict__ inverse) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i0 < N; i0 += stride * UG1) {
        uint32_t d[UG1], u[UG1];
#pragma unroll
        for (int q = 0; q < UG1; q++) {
            const int64_t i = i0 + q * stride;
            d[q] = i < N ? dest1[i] : 0u;
        }
#pragma unroll
        for (int q = 0; q < UG1; q++) {
            const int64_t i = i0 + q * stride;
            u[q] = i < N ? U1v[d[q]] : 0u;
        }
#pragma unroll
        for (int q = 0; q < UG1; q++) {
            const int64_t i = i0 + q * stride;
            if (i < N) inverse[i] = (IDX)u[q];
        }
    }
}

// Optional per-kernel timing (diagnostics): while enabled, every call records
// a CUDA event on its own stream before its first kernel and after each
// phase; the elapsed times of up to TIMED_CALLS calls are summed on query.
constexpr int NPHASE = 8;
constexpr int TIMED_CALLS = 64;
const char *const PHASE_NAME[NPHASE] = {"sample+splitters", "hist1",      "scatter1",
                                        "level2",           "leaf_dedup", "compact_unique",
                                        "unscatter2",       "unscatter1"};
struct PhaseTimer {
    std::mutex mu;
    bool on = false;
    bool created = false;
    int dev = -1;
    int calls = 0;
    cudaEvent_t ev[TIMED_CALLS][NPHASE + 1];
};
PhaseTimer g_timer;

// the event row of this call, or nullptr when timing is off or full
cudaEvent_t *timer_row() {
    std::lock_guard<std::mutex> lk(g_timer.mu);
    int dev = 0;
    cudaGetDevice(&dev);
    if (!g_timer.on || !g_timer.created || dev != g_timer.dev || g_timer.calls >= TIMED_CALLS)
        return nullptr;
    return g_timer.ev[g_timer.calls++];
}

inline void mark(cudaEvent_t *row, int i, cudaStream_t st) {
    if (row) cudaEventRecord(row[i], st);
}

template <int W>
cusci_status run(const Plan &p, const uint64_t *keys, unsigned char *ws, uint64_t *unique,
                 void *inverse, int index_bytes, int64_t *d_n_unique, int32_t *status,
                 cudaStream_t st) {
    using namespace radix;
    uint64_t *bt = (uint64_t *)(ws + p.o_bt);
    Key<1> *samp = (Key<1> *)(ws + p.o_samp), *samp2 = (Key<1> *)(ws + p.o_samp2);
    uint32_t *sidx = (uint32_t *)(ws + p.o_sidx), *sidx2 = (uint32_t *)(ws + p.o_sidx2);
    uint32_t *shist = (uint32_t *)(ws + p.o_shist);
    int64_t *sbase = (int64_t *)(ws + p.o_sbase);
    int64_t *scanws = (int64_t *)(ws + p.o_scanws);
    uint64_t *LS = (uint64_t *)(ws + p.o_LS);
    uint32_t *H1 = (uint32_t *)(ws + p.o_H1);
    int64_t *base1 = (int64_t *)(ws + p.o_base1);
    uint16_t *bid1 = (uint16_t *)(ws + p.o_bid1);
    uint64_t *K1 = (uint64_t *)(ws + p.o_K1);
    uint32_t *dest1 = (uint32_t *)(ws + p.o_dest1);
    Bid2 *bid2 = (Bid2 *)(ws + p.o_bid2);
    uint64_t *K2 = (uint64_t *)(ws + p.o_K2);
    uint32_t *dest2 = (uint32_t *)(ws + p.o_dest2);
    uint32_t *U2 = (uint32_t *)(ws + p.o_U2);
    uint64_t *tmpU = (uint64_t *)(ws + p.o_tmpU);
    int64_t *leafst = (int64_t *)(ws + p.o_leafst);
    int64_t *ucnt = (int64_t *)(ws + p.o_ucnt);
    int64_t *ubase = (int64_t *)(ws + p.o_ubase);
    const int sms = sm_count();
    int launches = 0;
    cudaEvent_t *tr = timer_row();
    mark(tr, 0, st);

    build_bt<<<1, 32, 0, st>>>(bt, p.n_bits, p.kcols);
    launches++;
    sample_keys<W><<<sms * 4, T, 0, st>>>(keys, p.N, p.NS, p.mode, p.n_bits, p.kcols, bt, (uint64_t *)samp,
                                          sidx);
    launches++;
    // sort the sample with the LSD building blocks
    {
        const size_t smem = sizeof(DownSmem<1>);
        cusci_status rc0 = allow_smem((const void *)downsweep<1>, smem, "dedup: smem attribute");
        if (rc0 != CUSCI_OK) return rc0;
        const int64_t nh = (int64_t)RADIX * p.gs;
        for (int pass = 0; pass < p.s_passes; pass++) {
            upsweep<1><<<p.gs, RT, 0, st>>>(samp, p.NS, pass * RBITS, p.gs_per, shist);
            widen_u32<<<64, 256, 0, st>>>(shist, nh, sbase);
            cusci_status rc = exclusive_scan_i64(sbase, nh, sbase, scanws, st);
            if (rc != CUSCI_OK) return rc;
            downsweep<1><<<p.gs, RT, smem, st>>>(samp, sidx, samp2, sidx2, p.NS, pass * RBITS,
                                                 p.gs_per, sbase);
            launches += 3;
            Key<1> *tk = samp; samp = samp2; samp2 = tk;
            uint32_t *ti = sidx; sidx = sidx2; sidx2 = ti;
        }
    }
    make_splitters<<<(int)((p.NL + 255) / 256), 256, 0, st>>>((const uint64_t *)samp, p.NS, p.NL,
                                                               LS);
    uint16_t *T1 = (uint16_t *)(ws + p.o_T1);
    uint64_t *krange = (uint64_t *)(ws + p.o_krange);
    build_T1<<<1, 1024, 0, st>>>((const uint64_t *)samp, p.NS, LS, p.B1, p.log2B1, T1, krange);
    launches++;
    launches++;
    // level 1
    const size_t sm_h1 = (size_t)p.B1 * 8 + (p.mode == 1 ? BT_MAX * 8 : 0) + (size_t)p.B1 * 4 +
                         ((size_t)(1 << LG_CELLS1) + 1) * 2;
    const size_t sm_x1 = (size_t)MAX_B1 * 4 + (p.mode == 1 ? BT_MAX * 8 : 0);
    {
        const char *what = "dedup: smem attribute";
        cusci_status rc0 = allow_smem((const void *)hist1<W>, (size_t)MAX_B1 * 12 + BT_MAX * 8 +
                                                                   ((size_t)(1 << LG_CELLS1) + 1) * 2,
                                      what);
        if (rc0 == CUSCI_OK)
            rc0 = allow_smem((const void *)scatter1<W>, (size_t)MAX_B1 * 4 + BT_MAX * 8, what);
        if (rc0 == CUSCI_OK) rc0 = allow_smem((const void *)leaf_dedup, sizeof(LeafSmem), what);
        if (rc0 != CUSCI_OK) return rc0;
    }
    mark(tr, 1, st);
    hist1<W><<<p.G, T, sm_h1, st>>>(keys, p.N, p.per_cta, p.mode, p.n_bits, p.n_ones, p.kcols, bt,
                                    LS, p.B1, p.log2B1, T1, krange, bid1, H1, status);
    mark(tr, 2, st);
    scatter1<W><<<p.G, T, sm_x1, st>>>(keys, p.N, p.per_cta, p.mode, p.n_bits, p.kcols, bt, bid1,
                                       p.B1, H1, base1, K1, dest1);
    cusci_status rc = CUSCI_OK;
    int64_t *kbase = (int64_t *)(ws + p.o_kbase);
    bucket_totals<<<(p.B1 + 255) / 256, 256, 0, st>>>(H1, p.G, p.B1, kbase);
    rc = exclusive_scan_i64(kbase, p.B1, kbase, scanws, st);
    if (rc != CUSCI_OK) return rc;
    launches += 3;
    mark(tr, 3, st);
    // level 2
    level2<<<p.B1, T, 0, st>>>(K1, p.N, base1, H1, p.G, p.B1, kbase, LS, p.NL, bid2, K2, dest2,
                               leafst);
    launches++;
    mark(tr, 4, st);
    // leaves
    uint32_t *pay = (uint32_t *)(ws + p.o_pay);
    leaf_dedup<<<sms * 4, T, sizeof(LeafSmem), st>>>(K2, K1, pay, p.N, p.NL, leafst, U2, tmpU, ucnt);
    launches++;
    mark(tr, 5, st);
    rc = exclusive_scan_i64(ucnt, p.NL, ubase, scanws, st);
    if (rc != CUSCI_OK) return rc;
    compact_unique<W><<<sms * 4, T, 0, st>>>(tmpU, leafst, ucnt, ubase, p.NL, p.mode, p.n_bits,
                                             p.n_ones, p.kcols, bt, unique, d_n_unique);
    mark(tr, 6, st);
    unscatter2<<<p.B1, T, 0, st>>>(base1, H1, p.G, p.B1, bid2, dest2, U2, ubase);
    mark(tr, 7, st);
    if (index_bytes == 4)
        unscatter1<int32_t><<<sms * 4, 256, 0, st>>>(dest1, dest2, p.N, (int32_t *)inverse);
    else
        unscatter1<int64_t><<<sms * 4, 256, 0, st>>>(dest1, dest2, p.N, (int64_t *)inverse);
    mark(tr, 8, st);
    launches += 3;
    CUSCI_LAUNCHED(launches, "sample-sort dedup");
    return CUSCI_OK;
}

}  // namespace ss

bool ss_eligible(int64_t N, int W, int n_bits, int n_ones) {
    int mode, kb;
    return ss::eligible(N, W, n_bits, n_ones, &mode, &kb);
}

size_t ss_workspace(int64_t N, int W, int n_bits, int n_ones) {
    int mode, kb;
    if (!ss::eligible(N, W, n_bits, n_ones, &mode, &kb)) return 0;
    return ss::make_plan(N, W, n_bits, n_ones, mode, kb).bytes;
}

cusci_status ss_dedup(const uint64_t *keys, int64_t N, int W, int n_bits, int n_ones, void *ws,
                      size_t ws_bytes, uint64_t *unique, void *inverse, int index_bytes,
                      int64_t *d_n_unique, int32_t *status, cudaStream_t st) {
    int mode, kb;
    if (!ss::eligible(N, W, n_bits, n_ones, &mode, &kb))
        return fail(CUSCI_ERR_INVALID, "dedup: sample-sort path not applicable");
    const ss::Plan p = ss::make_plan(N, W, n_bits, n_ones, mode, kb);
    if (ws_bytes < p.bytes)
        return fail(CUSCI_ERR_OOM, "cusci_dedup: workspace %zu < %zu bytes", ws_bytes, p.bytes);
    if (W == 1)
        return ss::run<1>(p, keys, (unsigned char *)ws, unique, inverse, index_bytes, d_n_unique,
                          status, st);
    return ss::run<2>(p, keys, (unsigned char *)ws, unique, inverse, index_bytes, d_n_unique,
                      status, st);
}

}  // namespace cusci

using namespace cusci;

extern "C" cusci_status cusci_set_kernel_timing(int on) {
    std::lock_guard<std::mutex> lk(ss::g_timer.mu);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cusci_set_kernel_timing: device");
    if (on && (!ss::g_timer.created || ss::g_timer.dev != dev)) {
        if (ss::g_timer.created) {
            for (int c = 0; c < ss::TIMED_CALLS; c++)
                for (int i = 0; i <= ss::NPHASE; i++) cudaEventDestroy(ss::g_timer.ev[c][i]);
            ss::g_timer.created = false;
        }
        for (int c = 0; c < ss::TIMED_CALLS; c++)
            for (int i = 0; i <= ss::NPHASE; i++) {
                e = cudaEventCreate(&ss::g_timer.ev[c][i]);
                if (e != cudaSuccess) return cuda_fail(e, "cusci_set_kernel_timing: events");
            }
        ss::g_timer.created = true;
        ss::g_timer.dev = dev;
    }
    ss::g_timer.on = on != 0;
    if (on) ss::g_timer.calls = 0;  // stopping keeps the record for the query
    return CUSCI_OK;
}

extern "C" const char *cusci_dedup_phase_name(int i) {
    return i >= 0 && i < ss::NPHASE ? ss::PHASE_NAME[i] : nullptr;
}

extern "C" int cusci_dedup_phase_ms(double *h_ms, int max, int *h_calls) {
    std::lock_guard<std::mutex> lk(ss::g_timer.mu);
    const int n = max < ss::NPHASE ? max : ss::NPHASE;
    for (int i = 0; i < n; i++) h_ms[i] = 0.0;
    int used = 0;
    for (int c = 0; ss::g_timer.created && c < ss::g_timer.calls; c++) {
        if (cudaEventSynchronize(ss::g_timer.ev[c][ss::NPHASE]) != cudaSuccess) {
            cudaGetLastError();  // a call that stopped early recorded no end event
            continue;
        }
        float t[ss::NPHASE];
        bool ok = true;
        for (int i = 0; i < ss::NPHASE && ok; i++)
            ok = cudaEventElapsedTime(&t[i], ss::g_timer.ev[c][i], ss::g_timer.ev[c][i + 1]) ==
                 cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            continue;
        }
        for (int i = 0; i < n; i++) h_ms[i] += t[i];
        used++;
    }
    if (h_calls) *h_calls = used;
    return n;
}
