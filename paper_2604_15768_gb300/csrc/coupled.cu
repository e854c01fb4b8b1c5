// Coupled-configuration generation: count pass, fill pass, source validation.
//
// Design (GB300 re-think of Algorithm 1, Sec. 4.2.2):
//  * one warp per source determinant, sources strided over a persistent grid;
//  * the determinant is decoded once into per-spin occupied / virtual strings
//    (spatial index = bit) and per-spin prefix-parity strings, so every
//    fermionic phase is a handful of bit tests (popc / ffs, no loops over bits);
//  * singles: lanes over the virtual orbital a, the element summed in the same
//    order as the closed form (h_ai, then +(ai|kk), -(ak|ki) for k ascending),
//    kept lanes compacted with a ballot;
//  * doubles: for each occupied pair (i, j) and virtual a the surviving b's are
//    one precomputed bitmask word (screening folded into the table, the "dual
//    screening" of Sec. 4.2.2), ANDed with the source's virtual string; lane b
//    finds its output slot by a popcount of the lower bits and reads its element
//    from the contiguous slab row T[pair][a][*] -- coalesced loads and stores;
//  * count-then-fill: the count pass computes |C_i| without writing, an
//    exclusive scan turns counts into CSR offsets, and the fill pass writes each
//    source's list into its own rows in canonical order (deterministic, no slab
//    atomics, unlike the g_counter reservation of Algorithm 1).
// All FP64 arithmetic uses explicit round-to-nearest intrinsics (no contraction),
// so elements are bit-identical to the closed forms summed in canonical order.

#include <stdlib.h>

#include "enumerate.cuh"

namespace cusci {
namespace {

using namespace enumr;
constexpr int WARPS_PER_BLOCK = 8;

template <int W>
struct FillEmit {
    uint64_t *__restrict__ out_d;
    double *__restrict__ out_h;
    int64_t beg, end;
    __device__ __forceinline__ bool pair_possible(const uint64_t (&)[W], int, int) const {
        return true;
    }
    __device__ __forceinline__ bool row_possible(const uint64_t (&)[W], int) const { return true; }
    __device__ __forceinline__ void operator()(const uint64_t (&t)[W], double h, int64_t rank) {
        const int64_t p = beg + rank;
        if (p < end) {
            if (W == 1) {
                out_d[p] = t[0];
            } else {
                reinterpret_cast<ulonglong2 *>(out_d)[p] = make_ulonglong2(t[0], t[W - 1]);
            }
            out_h[p] = h;
        }
    }
};

template <int W>
__global__ void __launch_bounds__(32 * WARPS_PER_BLOCK)
    count_kernel(SysView v, const uint64_t *__restrict__ dets, int64_t n, double eps,
                 int64_t *__restrict__ counts) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (int64_t)blockIdx.x * WARPS_PER_BLOCK + (threadIdx.x >> 5);
    const int64_t nwarps = (int64_t)gridDim.x * WARPS_PER_BLOCK;
    for (int64_t src = warp; src < n; src += nwarps) {
        Src<W> s;
        decode<W>(dets + src * W, v.norb, s);
        int64_t c = count_source<W>(v, s, eps, lane);
        if (lane == 0) counts[src] = c;
    }
}

template <int W, bool STAGE>
__global__ void __launch_bounds__(32 * WARPS_PER_BLOCK)
    fill_kernel(SysView v, const uint64_t *__restrict__ dets, int64_t n, double eps,
                const int64_t *__restrict__ offsets, uint64_t *__restrict__ out_d,
                double *__restrict__ out_h, int32_t *__restrict__ status) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    WarpStage st;
    WarpStage *stp = nullptr;
    if (STAGE) {
        stage_init(st, smem + (threadIdx.x >> 5) * stage_bytes(v.slab, v.mrow), v.slab, v.mrow,
                   lane, status);
        stp = &st;
    }
    const int64_t warp = (int64_t)blockIdx.x * WARPS_PER_BLOCK + (threadIdx.x >> 5);
    const int64_t nwarps = (int64_t)gridDim.x * WARPS_PER_BLOCK;
    for (int64_t src = warp; src < n; src += nwarps) {
        Src<W> s;
        decode<W>(dets + src * W, v.norb, s);
        const int64_t beg = offsets[src], end = offsets[src + 1];
        bool ok = end >= beg;
        if (ok) {
            FillEmit<W> em{out_d, out_h, beg, end};
            ok = visit_source<W>(v, s, eps, lane, em, stp) == end - beg;
        }
        if (!ok && lane == 0 && status) *status = CUSCI_ERR_OVERFLOW;
    }
}

__global__ void check_kernel(const uint64_t *__restrict__ dets, int64_t n, int W, int norb,
                             int na, int nb, int32_t *__restrict__ status) {
    const int M = 2 * norb;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        int ca = 0, cb = 0;
        bool bad = false;
        for (int w = 0; w < W; w++) {
            uint64_t x = dets[k * W + w];
            int hi = M - 64 * w;
            uint64_t keep = hi >= 64 ? ~0ull : (hi <= 0 ? 0ull : ((1ull << hi) - 1));
            if (x & ~keep) bad = true;
            x &= keep;
            ca += __popcll(x & 0x5555555555555555ull);
            cb += __popcll(x & 0xAAAAAAAAAAAAAAAAull);
        }
        if (bad || ca != na || cb != nb) *status = CUSCI_ERR_INVALID;
    }
}

int grid_for(int64_t n, int per_sm = 8) {
    int64_t want = (n + WARPS_PER_BLOCK - 1) / WARPS_PER_BLOCK;
    int64_t cap = (int64_t)sm_count() * per_sm;
    return (int)(want < cap ? (want < 1 ? 1 : want) : cap);
}

// Whether the fill stages each occupied pair's integral slab in shared memory
// by bulk copies (W = 1 only).  Off by default: on GB300 the unstaged form,
// whose slab reads hit L1/L2 at four times the occupancy (64 instead of 16
// warps per SM), measured 13.4 ms against 16.6 ms on the 100k-source mid
// workload.  CUSCI_FILL_STAGE=1 in the environment selects the staged form
// (identical results).
bool fill_stage_default() {
    static int v = -1;
    if (v < 0) {
        const char *e = getenv("CUSCI_FILL_STAGE");
        v = (e && e[0] == '1') ? 1 : 0;
    }
    return v == 1;
}

// fill launch: staged integral slabs in shared memory when they fit
template <int W>
cusci_status launch_fill(const SysView &v, const uint64_t *d_dets, int64_t n, double eps,
                         const int64_t *d_offsets, uint64_t *d_out_dets, double *d_out_h,
                         int32_t *d_status, cudaStream_t st) {
    const size_t smem = (size_t)WARPS_PER_BLOCK * stage_bytes(v.slab, v.mrow);
    if (W == 1 && smem <= 200 * 1024 && fill_stage_default()) {
        cusci_status rc = allow_smem((const void *)fill_kernel<W, true>, smem,
                                     "fill: shared-memory attribute");
        if (rc != CUSCI_OK) return rc;
        int per_sm = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &per_sm, fill_kernel<W, true>, 32 * WARPS_PER_BLOCK, smem);
        if (e != cudaSuccess || per_sm < 1) per_sm = 1;
        fill_kernel<W, true><<<grid_for(n, per_sm), 32 * WARPS_PER_BLOCK, smem, st>>>(
            v, d_dets, n, eps, d_offsets, d_out_dets, d_out_h, d_status);
    } else {
        fill_kernel<W, false><<<grid_for(n), 32 * WARPS_PER_BLOCK, 0, st>>>(
            v, d_dets, n, eps, d_offsets, d_out_dets, d_out_h, d_status);
    }
    CUSCI_LAUNCHED(1, "fill_kernel");
    return CUSCI_OK;
}

}  // namespace
}  // namespace cusci

using namespace cusci;

extern "C" cusci_status cusci_count_coupled(const cusci_system *sys, const uint64_t *d_dets,
                                            int64_t n, double eps, int64_t *d_counts,
                                            void *stream) {
    if (!sys) return fail(CUSCI_ERR_INVALID, "cusci_count_coupled: NULL system");
    if (n < 0) return fail(CUSCI_ERR_INVALID, "cusci_count_coupled: n < 0");
    if (n == 0) return CUSCI_OK;
    if (!d_dets || !d_counts) return fail(CUSCI_ERR_INVALID, "cusci_count_coupled: NULL buffer");
    if (eps != eps) return fail(CUSCI_ERR_INVALID, "cusci_count_coupled: eps is NaN");
    cudaStream_t st = (cudaStream_t)stream;
    const uint64_t *mask = NULL;
    cusci_status rc = masks_for(const_cast<cusci_system *>(sys), eps, st, &mask);
    if (rc != CUSCI_OK) return rc;
    SysView v = view_of(sys, mask);
    if (sys->W == 1)
        count_kernel<1><<<grid_for(n), 32 * WARPS_PER_BLOCK, 0, st>>>(v, d_dets, n, eps, d_counts);
    else
        count_kernel<2><<<grid_for(n), 32 * WARPS_PER_BLOCK, 0, st>>>(v, d_dets, n, eps, d_counts);
    CUSCI_LAUNCHED(1, "count_kernel");
    return CUSCI_OK;
}

extern "C" cusci_status cusci_gen_coupled(const cusci_system *sys, const uint64_t *d_dets,
                                          int64_t n, double eps, const int64_t *d_offsets,
                                          uint64_t *d_out_dets, double *d_out_h,
                                          int32_t *d_status, void *stream) {
    if (!sys) return fail(CUSCI_ERR_INVALID, "cusci_gen_coupled: NULL system");
    if (n < 0) return fail(CUSCI_ERR_INVALID, "cusci_gen_coupled: n < 0");
    if (n == 0) return CUSCI_OK;
    if (!d_dets || !d_offsets || !d_out_dets || !d_out_h)
        return fail(CUSCI_ERR_INVALID, "cusci_gen_coupled: NULL buffer");
    if (eps != eps) return fail(CUSCI_ERR_INVALID, "cusci_gen_coupled: eps is NaN");
    if (sys->W == 2 && ((uintptr_t)d_out_dets & 15u))
        return fail(CUSCI_ERR_INVALID, "cusci_gen_coupled: W=2 output must be 16-byte aligned");
    if (((uintptr_t)d_out_dets & 7u) || ((uintptr_t)d_out_h & 7u) || ((uintptr_t)d_dets & 7u))
        return fail(CUSCI_ERR_INVALID, "cusci_gen_coupled: buffers must be 8-byte aligned");
    cudaStream_t st = (cudaStream_t)stream;
    const uint64_t *mask = NULL;
    cusci_status rc = masks_for(const_cast<cusci_system *>(sys), eps, st, &mask);
    if (rc != CUSCI_OK) return rc;
    SysView v = view_of(sys, mask);
    if (sys->W == 1)
        return launch_fill<1>(v, d_dets, n, eps, d_offsets, d_out_dets, d_out_h, d_status, st);
    return launch_fill<2>(v, d_dets, n, eps, d_offsets, d_out_dets, d_out_h, d_status, st);
}

extern "C" cusci_status cusci_check_dets(const cusci_system *sys, const uint64_t *d_dets,
                                         int64_t n, int32_t *d_status, void *stream) {
    if (!sys || !d_status) return fail(CUSCI_ERR_INVALID, "cusci_check_dets: NULL argument");
    if (n < 0) return fail(CUSCI_ERR_INVALID, "cusci_check_dets: n < 0");
    if (n == 0) return CUSCI_OK;
    if (!d_dets) return fail(CUSCI_ERR_INVALID, "cusci_check_dets: NULL dets");
    int blocks = (int)((n + 255) / 256);
    if (blocks > sm_count() * 8) blocks = sm_count() * 8;
    check_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>(d_dets, n, sys->W, sys->norb,
                                                           sys->n_alpha, sys->n_beta, d_status);
    CUSCI_LAUNCHED(1, "check_kernel");
    return CUSCI_OK;
}
