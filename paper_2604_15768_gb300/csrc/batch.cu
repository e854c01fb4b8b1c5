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
    unsigned int *d_counter;         // device [2]: work cursor of the count and fill launches
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
    const int grid = sm_count() * 8;
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
    b->masks.assign(n_systems, NULL);
    cudaError_t e = cudaMalloc(&b->d_views, sizeof(SysView) * n_systems);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_counter, 2 * sizeof(unsigned int));
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
