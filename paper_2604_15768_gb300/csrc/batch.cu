// Batched generation over many independent systems in one persistent launch.
//
// The batch holds, on the device, the view of every system (its integral
// tables and screening masks) and a work list of (system, first source,
// number of sources) items.  Warps of one persistent grid pull items from an
// atomic counter, largest estimated cost first, so systems of very uneven
// size (10..50 spatial orbitals, 1k..50k sources) share the GPU without a
// launch per system -- the persistent grid-stride form of Algorithm 1
// extended over systems.  Sources and targets are stored as two words for
// every system (one-word systems carry a zero high word), so one CSR layout
// covers the whole batch.  Every count/fill launch is a fixed-size launch
// whose only host-side dependency is the batch object, so the sequence can be
// captured in a CUDA graph and replayed.

#include <algorithm>
#include <mutex>
#include <stdlib.h>
#include <string.h>
#include <vector>

#include "enumerate.cuh"

struct cusci_batch {
    int n_sys;
    std::vector<const cusci_system *> systems;
    std::vector<int64_t> src_begin;  // n_sys + 1, global source index of each system
    double eps;                      // eps the masks below were built for (NaN: none)
    std::vector<uint64_t *> masks;   // device screening masks of every system, owned by the
                                     // batch (graph replays never see another call's eps)
    cusci::SysView *d_views;         // device [n_sys]
    int4 *d_items;                   // device work list: (system, first, count, unused)
    int n_items;
    int chunk;
    int blocks_per_sm;               // persistent grid: blocks per SM of the count/fill launches
    unsigned int *d_counter;         // device [2]: work cursor of the count and fill launches
    // batched de-duplication: per system its spin-orbital count M and electron
    // count (device int2[n_sys]) and the base of its rank range in the joint
    // key space (device uint64[n_sys + 1]; base[n_sys] = size of that space)
    int2 *d_sysinfo;
    int max_bits = 0, max_ones = 0;  // over the systems: M and n_alpha + n_beta
    uint64_t *d_base;
    int64_t *d_src_begin;            // device copy of src_begin (first dedup call)
    bool d_src_begin_ready;
    uint64_t space;                  // sum of C(M_k, n_k); 0 if it does not fit 64 bits
    int key_bits;
};

namespace cusci {
namespace {

using namespace enumr;
constexpr int BW = 8;  // warps per block

struct BatchFill {
    uint64_t *__restrict__ out_d;
    double *__restrict__ out_h;
    int64_t beg, end;
    template <int W>
    __device__ __forceinline__ void operator()(const uint64_t (&t)[W], double h, int64_t rank) {
        const int64_t p = beg + rank;
        if (p < end) {
            reinterpret_cast<ulonglong2 *>(out_d)[p] = make_ulonglong2(t[0], W == 2 ? t[W - 1] : 0ull);
            out_h[p] = h;
        }
    }
};

template <int W>
struct FillAdapter {
    BatchFill &f;
    __device__ __forceinline__ bool pair_possible(const uint64_t (&)[W], int, int) const {
        return true;
    }
    __device__ __forceinline__ bool row_possible(const uint64_t (&)[W], int) const { return true; }
    __device__ __forceinline__ void operator()(const uint64_t (&t)[W], double h, int64_t rank) {
        f.template operator()<W>(t, h, rank);
    }
};

template <int W, bool FILL>
__device__ void batch_source(const SysView &v, const uint64_t *__restrict__ det, double eps,
                             int lane, int64_t src, int64_t *__restrict__ counts,
                             const int64_t *__restrict__ offsets, uint64_t *__restrict__ out_d,
                             double *__restrict__ out_h, int32_t *__restrict__ status) {
    Src<W> s;
    decode<W>(det, v.norb, s);
    if (!FILL) {
        const int64_t c = count_source<W>(v, s, eps, lane);
        if (lane == 0) counts[src] = c;
    } else {
        const int64_t beg = offsets[src], end = offsets[src + 1];
        BatchFill f{out_d, out_h, beg, end};
        FillAdapter<W> em{f};
        const int64_t got = visit_source<W>(v, s, eps, lane, em);
        if (got != end - beg && lane == 0 && status) *status = CUSCI_ERR_OVERFLOW;
    }
}

template <bool FILL>
__global__ void __launch_bounds__(32 * BW)
    batch_kernel(const SysView *__restrict__ views, const int4 *__restrict__ items, int n_items,
                 unsigned int *__restrict__ cursor, const uint64_t *__restrict__ dets, double eps,
                 int64_t *__restrict__ counts, const int64_t *__restrict__ offsets,
                 uint64_t *__restrict__ out_d, double *__restrict__ out_h,
                 int32_t *__restrict__ status) {
    const int lane = threadIdx.x & 31;
    for (;;) {
        unsigned int it = 0;
        if (lane == 0) it = atomicAdd(cursor, 1u);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= (unsigned)n_items) break;
        const int4 w = items[it];
        const SysView v = views[w.x];
        for (int64_t src = w.y; src < (int64_t)w.y + w.z; src++) {
            const uint64_t *det = dets + src * 2;
            if (v.W == 1)
                batch_source<1, FILL>(v, det, eps, lane, src, counts, offsets, out_d, out_h, status);
            else
                batch_source<2, FILL>(v, det, eps, lane, src, counts, offsets, out_d, out_h, status);
        }
    }
}

int64_t structural(const cusci_system *s) {
    const int64_t n = s->norb, a = s->n_alpha, b = s->n_beta, va = n - a, vb = n - b;
    return 1 + a * va + b * vb + a * (a - 1) / 2 * (va * (va - 1) / 2) +
           b * (b - 1) / 2 * (vb * (vb - 1) / 2) + a * va * b * vb;
}

cusci_status build_items(cusci_batch *b, int chunk) {
    std::vector<int4> items;
    std::vector<int64_t> cost;
    for (int k = 0; k < b->n_sys; k++) {
        const int64_t per = structural(b->systems[k]);
        for (int64_t s = b->src_begin[k]; s < b->src_begin[k + 1]; s += chunk) {
            const int64_t c = std::min<int64_t>(chunk, b->src_begin[k + 1] - s);
            items.push_back(make_int4(k, (int)s, (int)c, 0));
            cost.push_back(per * c);
        }
    }
    std::vector<size_t> order(items.size());
    for (size_t i = 0; i < order.size(); i++) order[i] = i;
    std::stable_sort(order.begin(), order.end(),
                     [&](size_t x, size_t y) { return cost[x] > cost[y]; });
    std::vector<int4> sorted(items.size());
    for (size_t i = 0; i < order.size(); i++) sorted[i] = items[order[i]];
    cudaFree(b->d_items);
    b->d_items = NULL;
    b->n_items = (int)sorted.size();
    b->chunk = chunk;
    if (b->n_items == 0) return CUSCI_OK;
    cudaError_t e = cudaMalloc(&b->d_items, sizeof(int4) * sorted.size());
    if (e == cudaSuccess)
        e = cudaMemcpy(b->d_items, sorted.data(), sizeof(int4) * sorted.size(),
                       cudaMemcpyHostToDevice);
    return e == cudaSuccess ? CUSCI_OK : cuda_fail(e, "batch: work list");
}

cusci_status refresh_views(cusci_batch *b, double eps, cudaStream_t st) {
    uint64_t want, have;
    memcpy(&want, &eps, 8);
    memcpy(&have, &b->eps, 8);
    if (want == have) return CUSCI_OK;
    // the previous launches may still read the masks being rebuilt
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "batch: drain before rebuilding masks");
    std::vector<SysView> views(b->n_sys);
    for (int k = 0; k < b->n_sys; k++) {
        cusci_status rc = build_masks_into(b->systems[k], eps, st, b->masks[k]);
        if (rc != CUSCI_OK) return rc;
        views[k] = view_of(b->systems[k], b->masks[k]);
    }
    e = cudaMemcpyAsync(b->d_views, views.data(), sizeof(SysView) * b->n_sys,
                        cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "batch: views");
    b->eps = eps;
    return CUSCI_OK;
}

cusci_status launch(cusci_batch *b, bool fill, const uint64_t *d_dets, double eps,
                    int64_t *d_counts, const int64_t *d_offsets, uint64_t *d_out, double *d_h,
                    int32_t *d_status, cudaStream_t st) {
    cusci_status rc = refresh_views(b, eps, st);
    if (rc != CUSCI_OK) return rc;
    if (b->n_items == 0) return CUSCI_OK;
    unsigned int *cur = b->d_counter + (fill ? 1 : 0);
    cudaError_t e = cudaMemsetAsync(cur, 0, sizeof(unsigned int), st);
    if (e != cudaSuccess) return cuda_fail(e, "batch: cursor");
    const int grid = sm_count() * b->blocks_per_sm;
    if (fill)
        batch_kernel<true><<<grid, 32 * BW, 0, st>>>(b->d_views, b->d_items, b->n_items, cur,
                                                     d_dets, eps, d_counts, d_offsets, d_out, d_h,
                                                     d_status);
    else
        batch_kernel<false><<<grid, 32 * BW, 0, st>>>(b->d_views, b->d_items, b->n_items, cur,
                                                      d_dets, eps, d_counts, d_offsets, d_out,
                                                      d_h, d_status);
    CUSCI_LAUNCHED(1, "batch kernel");
    return CUSCI_OK;
}


// ---------------------------------------------------------------- batched de-duplication
// Every target of system k is mapped to base_k + its combinatorial rank among
// the C(M_k, n_k) determinants of that system (rank = sum over the set bits,
// in increasing position p with running count c = 1, 2, ..., of C(p, c)); the
// map is order preserving within a system and the systems' ranges are
// disjoint and ordered, so one de-duplication of these 64-bit keys yields
// every system's sorted distinct set, contiguous and in system order.

__device__ uint64_t g_bbinom[128 * 65];  // C(m, c) for m < 128, c <= 64 (saturated)
std::mutex g_bbinom_mu;
bool g_bbinom_ready[64] = {false};

unsigned __int128 binom_u128(int m, int k) {
    if (k < 0 || k > m) return 0;
    unsigned __int128 r = 1;
    for (int i = 1; i <= k; i++) r = r * (unsigned)(m - k + i) / (unsigned)i;
    return r;
}

cusci_status ensure_bbinom() {
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return fail(CUSCI_ERR_INVALID, "batch: device id out of range");
    std::lock_guard<std::mutex> lk(g_bbinom_mu);
    if (g_bbinom_ready[dev]) return CUSCI_OK;
    static uint64_t host[128 * 65];
    for (int m = 0; m < 128; m++)
        for (int c = 0; c <= 64; c++) {
            const unsigned __int128 v = binom_u128(m, c);
            host[m * 65 + c] = v > (unsigned __int128)~0ull ? ~0ull : (uint64_t)v;
        }
    cudaError_t e = cudaMemcpyToSymbol(g_bbinom, host, sizeof(host));
    if (e != cudaSuccess) return cuda_fail(e, "batch: binomial table");
    g_bbinom_ready[dev] = true;
    return CUSCI_OK;
}

// largest k with v[k] <= x over v[0..n] (v ascending, v[0] <= x)
__device__ __forceinline__ int seg_of(const int64_t *v, int n, int64_t x) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (v[mid] <= x) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// entry begins of the systems: ebeg[k] = offsets[src_begin[k]]
__global__ void bd_ebeg(const int64_t *__restrict__ offsets, const int64_t *__restrict__ src_begin,
                        int n_sys, int64_t *__restrict__ ebeg) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k <= n_sys) ebeg[k] = offsets[src_begin[k]];
}

// Shared-memory copies for the rank kernels: C(m, c) for m < bm, c < bk at
// [m * bk + c], and the n_sys + 1 system boundaries of the index being
// searched.  Staged when they fit in BD_SMEM bytes (else read from global).
constexpr size_t BD_SMEM = 48 * 1024;

size_t bd_smem_bytes(int bm, int bk, int n_sys) {
    const size_t b = (size_t)bm * bk * 8 + (size_t)(n_sys + 1) * 8;
    return b <= BD_SMEM ? b : 0;
}

struct BdTables {
    const uint64_t *binom;  // [m * stride + c]
    int stride;
    const int64_t *bounds;  // n_sys + 1 system boundaries
};

__device__ BdTables bd_stage(bool staged, int bm, int bk, int n_sys,
                             const int64_t *__restrict__ bounds) {
    extern __shared__ __align__(16) unsigned char bdsm[];
    if (!staged) return BdTables{g_bbinom, 65, bounds};
    uint64_t *sb = reinterpret_cast<uint64_t *>(bdsm);
    int64_t *sbd = reinterpret_cast<int64_t *>(bdsm + (size_t)bm * bk * 8);
    for (int i = threadIdx.x; i < bm * bk; i += blockDim.x) {
        const int m = i / bk, c = i - m * bk;
        sb[i] = g_bbinom[m * 65 + c];
    }
    for (int i = threadIdx.x; i <= n_sys; i += blockDim.x) sbd[i] = bounds[i];
    __syncthreads();
    return BdTables{sb, bk, sbd};
}

__global__ void bd_keys(const uint64_t *__restrict__ tgt, int64_t total,
                        const int64_t *__restrict__ ebeg, int n_sys,
                        const int2 *__restrict__ info, const uint64_t *__restrict__ base,
                        uint64_t *__restrict__ keys, int32_t *__restrict__ status, int staged,
                        int bm, int bk) {
    const BdTables tb = bd_stage(staged != 0, bm, bk, n_sys, ebeg);
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int k = seg_of(tb.bounds, n_sys + 1, e);
        const int2 in = info[k];
        uint64_t r = 0;
        int c = 0;
        bool bad = false;
#pragma unroll
        for (int w = 0; w < 2; w++) {
            uint64_t x = tgt[2 * e + w];
            const int hi = in.x - 64 * w;
            const uint64_t keep = hi >= 64 ? ~0ull : (hi <= 0 ? 0ull : ((1ull << hi) - 1));
            if (x & ~keep) bad = true;
            for (x &= keep; x; x &= x - 1) {
                const int pos = 64 * w + __ffsll((long long)x) - 1;
                c++;
                if (c < tb.stride) r += tb.binom[pos * tb.stride + c];
            }
        }
        if ((bad || c != in.y) && status) *status = CUSCI_ERR_INVALID;
        keys[e] = base[k] + r;
    }
}

// first distinct index of every system: ub[k] = number of distinct keys < base[k]
__global__ void bd_bounds(const uint64_t *__restrict__ uniq, const int64_t *__restrict__ d_nu,
                          const uint64_t *__restrict__ base, int n_sys, int64_t *__restrict__ ub,
                          int64_t *__restrict__ n_unique) {
    const int k = threadIdx.x;  // one block
    const int64_t nu = *d_nu;
    if (k <= n_sys) {
        int64_t lo = 0, hi = nu;
        if (k == n_sys) {
            lo = nu;
        } else {
            const uint64_t x = base[k];
            while (lo < hi) {
                const int64_t mid = (lo + hi) >> 1;
                if (uniq[mid] < x) lo = mid + 1;
                else hi = mid;
            }
        }
        ub[k] = lo;
    }
    __syncthreads();
    if (k < n_sys) n_unique[k] = ub[k + 1] - ub[k];
}

// distinct keys back to determinants, at each system's entry range
__global__ void bd_unrank(const uint64_t *__restrict__ uniq, const int64_t *__restrict__ d_nu,
                          const int64_t *__restrict__ ub, const int64_t *__restrict__ ebeg,
                          int n_sys, const int2 *__restrict__ info,
                          const uint64_t *__restrict__ base, uint64_t *__restrict__ out,
                          int staged, int bm, int bk) {
    const BdTables tb = bd_stage(staged != 0, bm, bk, n_sys, ub);
    const int64_t nu = *d_nu;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < nu;
         j += (int64_t)gridDim.x * blockDim.x) {
        const int k = seg_of(tb.bounds, n_sys + 1, j);
        const int2 in = info[k];
        uint64_t v = uniq[j] - base[k];
        uint64_t d0 = 0ull, d1 = 0ull;  // two words held in registers
        int p = in.x - 1;
        for (int c = in.y; c >= 1; c--) {
            while (p >= c && tb.binom[p * tb.stride + c] > v) p--;
            if (p >= c) v -= tb.binom[p * tb.stride + c];
            if (p >= 64) d1 |= 1ull << (p - 64);
            else if (p >= 0) d0 |= 1ull << p;
            p--;
        }
        const int64_t at = ebeg[k] + (j - tb.bounds[k]);
        out[2 * at] = d0;
        out[2 * at + 1] = d1;
    }
}

// global distinct ids to ids within each system
__global__ void bd_localize(int32_t *__restrict__ inv, int64_t total,
                            const int64_t *__restrict__ ebeg, int n_sys,
                            const int64_t *__restrict__ ub) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int k = seg_of(ebeg, n_sys + 1, e);
        inv[e] = (int32_t)(inv[e] - ub[k]);
    }
}

size_t bd_al(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace
}  // namespace cusci

using namespace cusci;

extern "C" cusci_status cusci_batch_create(const cusci_system *const *systems, int n_systems,
                                           const int64_t *h_sources, int chunk,
                                           cusci_batch **out) {
    if (!out || !systems || !h_sources || n_systems < 1 || chunk < 1)
        return fail(CUSCI_ERR_INVALID, "cusci_batch_create: bad argument");
    *out = NULL;
    cusci_batch *b = new (std::nothrow) cusci_batch();
    if (!b) return fail(CUSCI_ERR_OOM, "cusci_batch_create: host allocation");
    b->n_sys = n_systems;
    b->systems.assign(systems, systems + n_systems);
    b->src_begin.assign(n_systems + 1, 0);
    for (int k = 0; k < n_systems; k++) {
        if (!systems[k] || h_sources[k] < 0) {
            delete b;
            return fail(CUSCI_ERR_INVALID, "cusci_batch_create: system %d invalid", k);
        }
        b->src_begin[k + 1] = b->src_begin[k] + h_sources[k];
    }
    if (b->src_begin[n_systems] >= ((int64_t)1 << 31)) {
        delete b;
        return fail(CUSCI_ERR_UNSUPPORTED, "cusci_batch_create: more than 2^31 sources");
    }
    b->eps = __builtin_nan("");
    b->d_views = NULL;
    b->d_items = NULL;
    b->d_counter = NULL;
    b->d_sysinfo = NULL;
    b->d_base = NULL;
    b->d_src_begin = NULL;
    b->d_src_begin_ready = false;
    b->blocks_per_sm = 8;
    b->masks.assign(n_systems, NULL);
    // joint key space of the batched de-duplication
    std::vector<int2> info(n_systems);
    std::vector<uint64_t> base(n_systems + 1, 0);
    bool fits = true;
    for (int k = 0; k < n_systems; k++) {
        info[k] = make_int2(systems[k]->M, systems[k]->n_alpha + systems[k]->n_beta);
        if (info[k].x > b->max_bits) b->max_bits = info[k].x;
        if (info[k].y > b->max_ones) b->max_ones = info[k].y;
        const unsigned __int128 c = binom_u128(info[k].x, info[k].y);
        const unsigned __int128 nb = (unsigned __int128)base[k] + c;
        if (c > (unsigned __int128)~0ull || nb > (unsigned __int128)~0ull) fits = false;
        base[k + 1] = fits ? (uint64_t)nb : 0ull;
    }
    b->space = fits ? base[n_systems] : 0ull;
    b->key_bits = 1;
    while (b->key_bits < 64 && (b->space - 1) >> b->key_bits) b->key_bits++;
    cudaError_t e = cudaMalloc(&b->d_views, sizeof(SysView) * n_systems);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_counter, 2 * sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_sysinfo, sizeof(int2) * n_systems);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_base, sizeof(uint64_t) * (n_systems + 1));
    if (e == cudaSuccess)
        e = cudaMemcpy(b->d_sysinfo, info.data(), sizeof(int2) * n_systems, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(b->d_base, base.data(), sizeof(uint64_t) * (n_systems + 1),
                       cudaMemcpyHostToDevice);
    for (int k = 0; k < n_systems && e == cudaSuccess; k++)
        e = cudaMalloc(&b->masks[k], mask_words(systems[k]) * sizeof(uint64_t));
    if (e != cudaSuccess) {
        cusci_batch_destroy(b);
        return cuda_fail(e, "cusci_batch_create: cudaMalloc");
    }
    cusci_status rc = build_items(b, chunk);
    if (rc != CUSCI_OK) {
        cusci_batch_destroy(b);
        return rc;
    }
    *out = b;
    return CUSCI_OK;
}

extern "C" void cusci_batch_destroy(cusci_batch *b) {
    if (!b) return;
    cudaFree(b->d_views);
    cudaFree(b->d_items);
    cudaFree(b->d_counter);
    cudaFree(b->d_sysinfo);
    cudaFree(b->d_base);
    cudaFree(b->d_src_begin);
    for (uint64_t *m : b->masks) cudaFree(m);
    delete b;
}

extern "C" cusci_status cusci_batch_set_chunk(cusci_batch *b, int chunk) {
    if (!b || chunk < 1) return fail(CUSCI_ERR_INVALID, "cusci_batch_set_chunk: bad argument");
    return build_items(b, chunk);
}

extern "C" int64_t cusci_batch_sources(const cusci_batch *b) {
    return b ? b->src_begin[b->n_sys] : 0;
}

extern "C" cusci_status cusci_batch_count(cusci_batch *b, const uint64_t *d_dets, double eps,
                                          int64_t *d_counts, void *stream) {
    if (!b || !d_dets || !d_counts) return fail(CUSCI_ERR_INVALID, "cusci_batch_count: NULL");
    if (eps != eps) return fail(CUSCI_ERR_INVALID, "cusci_batch_count: eps is NaN");
    return launch(b, false, d_dets, eps, d_counts, NULL, NULL, NULL, NULL, (cudaStream_t)stream);
}

extern "C" cusci_status cusci_batch_gen(cusci_batch *b, const uint64_t *d_dets, double eps,
                                        const int64_t *d_offsets, uint64_t *d_out_dets,
                                        double *d_out_h, int32_t *d_status, void *stream) {
    if (!b || !d_dets || !d_offsets || !d_out_dets || !d_out_h)
        return fail(CUSCI_ERR_INVALID, "cusci_batch_gen: NULL");
    if (eps != eps) return fail(CUSCI_ERR_INVALID, "cusci_batch_gen: eps is NaN");
    if (((uintptr_t)d_out_dets & 15u) || ((uintptr_t)d_out_h & 7u))
        return fail(CUSCI_ERR_INVALID, "cusci_batch_gen: outputs misaligned");
    return launch(b, true, d_dets, eps, NULL, d_offsets, d_out_dets, d_out_h, d_status,
                  (cudaStream_t)stream);
}

extern "C" cusci_status cusci_batch_set_grid(cusci_batch *b, int blocks_per_sm) {
    if (!b || blocks_per_sm < 1 || blocks_per_sm > 32)
        return fail(CUSCI_ERR_INVALID, "cusci_batch_set_grid: bad argument");
    b->blocks_per_sm = blocks_per_sm;
    return CUSCI_OK;
}

extern "C" cusci_status cusci_batch_dedup_workspace(const cusci_batch *b, int64_t total,
                                                    size_t *bytes) {
    if (!b || !bytes || total < 0)
        return fail(CUSCI_ERR_INVALID, "cusci_batch_dedup_workspace: bad argument");
    if (b->space == 0)
        return fail(CUSCI_ERR_UNSUPPORTED, "cusci_batch_dedup: joint key space exceeds 64 bits");
    size_t inner = 0;
    cusci_status rc = cusci_dedup_workspace(total > 0 ? total : 1, 1, b->key_bits, -1, &inner);
    if (rc != CUSCI_OK) return rc;
    const size_t t = (size_t)(total > 0 ? total : 1);
    *bytes = bd_al(t * 8) * 2 + bd_al(((size_t)b->n_sys + 1) * 8) * 2 + bd_al(8) + bd_al(inner);
    return CUSCI_OK;
}

extern "C" cusci_status cusci_batch_dedup(cusci_batch *b, const int64_t *d_offsets,
                                          const uint64_t *d_targets, int64_t total, void *d_ws,
                                          size_t ws_bytes, uint64_t *d_unique, int32_t *d_inverse,
                                          int64_t *d_n_unique, int32_t *d_status, void *stream) {
    if (!b || !d_offsets || (total > 0 && (!d_targets || !d_unique || !d_inverse)) || !d_n_unique)
        return fail(CUSCI_ERR_INVALID, "cusci_batch_dedup: bad argument");
    if (total >= ((int64_t)1 << 31))
        return fail(CUSCI_ERR_UNSUPPORTED, "cusci_batch_dedup: int32 ids need fewer than 2^31 entries");
    size_t need = 0;
    cusci_status rc = cusci_batch_dedup_workspace(b, total, &need);
    if (rc != CUSCI_OK) return rc;
    if (!d_ws || ws_bytes < need || ((uintptr_t)d_ws & 255u))
        return fail(CUSCI_ERR_OOM, "cusci_batch_dedup: workspace %zu < %zu bytes (or misaligned)",
                    ws_bytes, need);
    rc = ensure_bbinom();
    if (rc != CUSCI_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const int ns = b->n_sys;
    if (total == 0) {
        cudaError_t e = cudaMemsetAsync(d_n_unique, 0, sizeof(int64_t) * ns, st);
        return e == cudaSuccess ? CUSCI_OK : cuda_fail(e, "cusci_batch_dedup: memset");
    }
    unsigned char *w = (unsigned char *)d_ws;
    const size_t t = (size_t)total;
    uint64_t *keys = (uint64_t *)w; w += bd_al(t * 8);
    uint64_t *uniq = (uint64_t *)w; w += bd_al(t * 8);
    int64_t *ebeg = (int64_t *)w; w += bd_al(((size_t)ns + 1) * 8);
    int64_t *ub = (int64_t *)w; w += bd_al(((size_t)ns + 1) * 8);
    int64_t *d_nu = (int64_t *)w; w += bd_al(8);
    void *inner = w;
    const size_t inner_bytes = ws_bytes - (size_t)(w - (unsigned char *)d_ws);
    // source begins of the systems, on the device once
    if (!b->d_src_begin_ready) {
        cudaError_t e = cudaMalloc(&b->d_src_begin, sizeof(int64_t) * (ns + 1));
        if (e == cudaSuccess)
            e = cudaMemcpy(b->d_src_begin, b->src_begin.data(), sizeof(int64_t) * (ns + 1),
                           cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(e, "cusci_batch_dedup: source begins");
        b->d_src_begin_ready = true;
    }
    int blocks = (int)((total + 255) / 256);
    if (blocks > sm_count() * 8) blocks = sm_count() * 8;
    bd_ebeg<<<1, 128 * ((ns + 128) / 128), 0, st>>>(d_offsets, b->d_src_begin, ns, ebeg);
    // binomial rows up to the largest M and electron count of the batch
    const int bm = b->max_bits, bk = b->max_ones + 1;
    const size_t bsm = bd_smem_bytes(bm, bk, ns);
    bd_keys<<<blocks, 256, bsm, st>>>(d_targets, total, ebeg, ns, b->d_sysinfo, b->d_base, keys,
                                      d_status, bsm > 0 ? 1 : 0, bm, bk);
    CUSCI_LAUNCHED(2, "batched dedup keys");
    rc = cusci_dedup(keys, total, 1, b->key_bits, -1, inner, inner_bytes, uniq, d_inverse, 4, d_nu,
                     NULL, d_status, stream);
    if (rc != CUSCI_OK) return rc;
    bd_bounds<<<1, 128 * ((ns + 128) / 128), 0, st>>>(uniq, d_nu, b->d_base, ns, ub, d_n_unique);
    bd_unrank<<<blocks, 256, bsm, st>>>(uniq, d_nu, ub, ebeg, ns, b->d_sysinfo, b->d_base,
                                        d_unique, bsm > 0 ? 1 : 0, bm, bk);
    bd_localize<<<blocks, 256, 0, st>>>(d_inverse, total, ebeg, ns, ub);
    CUSCI_LAUNCHED(3, "batched dedup split");
    return CUSCI_OK;
}
