// Enumeration of the coupled set of one source determinant by one warp, shared
// by the count / fill passes and the energy kernels so that every consumer
// visits exactly the same entries in exactly the same canonical order.
#pragma once

#include "cusci_internal.cuh"

namespace cusci {
namespace enumr {

constexpr unsigned FULL = 0xffffffffu;


__device__ __forceinline__ uint64_t compact_even(uint64_t x) {
    x &= 0x5555555555555555ull;
    x = (x | (x >> 1)) & 0x3333333333333333ull;
    x = (x | (x >> 2)) & 0x0F0F0F0F0F0F0F0Full;
    x = (x | (x >> 4)) & 0x00FF00FF00FF00FFull;
    x = (x | (x >> 8)) & 0x0000FFFF0000FFFFull;
    x = (x | (x >> 16)) & 0x00000000FFFFFFFFull;
    return x;
}

__device__ __forceinline__ uint64_t prefix_xor(uint64_t x) {
    x ^= x << 1;
    x ^= x << 2;
    x ^= x << 4;
    x ^= x << 8;
    x ^= x << 16;
    x ^= x << 32;
    return x;
}

__device__ __forceinline__ double flip_sign(double v, uint32_t odd) {
    return __longlong_as_double(__double_as_longlong(v) ^ ((unsigned long long)(odd & 1u) << 63));
}

template <int W>
struct Src {
    uint64_t d[W];    // determinant, bits at or above M cleared
    uint64_t occ[2];  // per spin: bit p set iff spin orbital 2p+sigma occupied
    uint64_t vir[2];  // per spin: complement within norb
    uint64_t par[2];  // per spin: bit p = parity of occupied spin orbitals below 2p+sigma
};

template <int W>
__device__ __forceinline__ void decode(const uint64_t *__restrict__ det, int norb, Src<W> &s) {
    const int M = 2 * norb;
    uint64_t carry = 0;
    uint64_t ex[W];
#pragma unroll
    for (int w = 0; w < W; w++) {
        uint64_t x = det[w];
        int hi = M - 64 * w;
        if (hi < 64) x &= (hi <= 0) ? 0ull : ((1ull << hi) - 1);
        s.d[w] = x;
        uint64_t px = prefix_xor(x);
        ex[w] = (px << 1) ^ carry;
        carry = ((px >> 63) & 1ull) ? ~carry : carry;
    }
    const uint64_t full = norb >= 64 ? ~0ull : ((1ull << norb) - 1);
#pragma unroll
    for (int sg = 0; sg < 2; sg++) {
        uint64_t o = compact_even(s.d[0] >> sg);
        uint64_t p = compact_even(ex[0] >> sg);
        if (W == 2) {
            o |= compact_even(s.d[W - 1] >> sg) << 32;
            p |= compact_even(ex[W - 1] >> sg) << 32;
        }
        s.occ[sg] = o;
        s.vir[sg] = ~o & full;
        s.par[sg] = p;
    }
}

// two-entry selects keep per-spin arrays in registers (no dynamic indexing)
__device__ __forceinline__ uint64_t sel2(const uint64_t (&x)[2], int k) { return k ? x[1] : x[0]; }
__device__ __forceinline__ uint32_t sel2(const uint32_t (&x)[2], int k) { return k ? x[1] : x[0]; }

__device__ __forceinline__ uint32_t par_bit(const uint64_t (&par)[2], int so) {
    return (uint32_t)((sel2(par, so & 1) >> (so >> 1)) & 1ull);
}

template <int W>
__device__ __forceinline__ void flip_bit(uint64_t (&d)[W], int so) {
#pragma unroll
    for (int w = 0; w < W; w++)
        if ((so >> 6) == w) d[w] ^= 1ull << (so & 63);
}

// Single excitation element before the phase: h_ai + sum_{k in O, k != i}
// [(ai|kk) - delta(spin k, spin a) (ak|ki)], k ascending in spin-orbital order.
template <int W>
__device__ __forceinline__ double single_value(const SysView &v, const Src<W> &s, int i, int pa) {
    const int n = v.norb, pi = i >> 1, sg = i & 1;
    const double *__restrict__ s1 = v.S1 + ((size_t)pa * n + pi) * n;
    const double *__restrict__ s2 = v.S2 + ((size_t)pa * n + pi) * n;
    double acc = __ldg(v.h1 + pa * n + pi);
#pragma unroll
    for (int w = 0; w < W; w++) {
        for (uint64_t r = s.d[w]; r; r &= r - 1) {
            int k = 64 * w + __ffsll((long long)r) - 1;
            if (k == i) continue;
            int pk = k >> 1;
            acc = __dadd_rn(acc, __ldg(s1 + pk));
            if ((k & 1) == sg) acc = __dsub_rn(acc, __ldg(s2 + pk));
        }
    }
    return acc;
}

// Diagonal element: (Ecore + sum_i h_ii) + sum_{i<j} [(ii|jj) - same-spin (ij|ji)].
template <int W>
__device__ __forceinline__ double diagonal_value(const SysView &v, const Src<W> &s) {
    const int n = v.norb;
    double e1 = 0.0, e2 = 0.0;
#pragma unroll
    for (int w = 0; w < W; w++)
        for (uint64_t r = s.d[w]; r; r &= r - 1) {
            int p = (64 * w + __ffsll((long long)r) - 1) >> 1;
            e1 = __dadd_rn(e1, __ldg(v.h1 + p * n + p));
        }
#pragma unroll
    for (int wi = 0; wi < W; wi++)
        for (uint64_t ri = s.d[wi]; ri; ri &= ri - 1) {
            int i = 64 * wi + __ffsll((long long)ri) - 1;
            int pi = i >> 1;
#pragma unroll
            for (int wj = 0; wj < W; wj++) {
                uint64_t rj = s.d[wj];
                if (wj < wi) rj = 0;
                else if (wj == wi) rj &= (i & 63) == 63 ? 0ull : (~0ull << ((i & 63) + 1));
                for (; rj; rj &= rj - 1) {
                    int j = 64 * wj + __ffsll((long long)rj) - 1;
                    int pj = j >> 1;
                    e2 = __dadd_rn(e2, __ldg(v.J + pi * n + pj));
                    if (((i ^ j) & 1) == 0) e2 = __dsub_rn(e2, __ldg(v.K + pi * n + pj));
                }
            }
        }
    return __dadd_rn(__dadd_rn(v.ecore, e1), e2);
}

__device__ __forceinline__ int lanes_below(uint32_t ballot, int lane) {
    return __popc(ballot & ((1u << lane) - 1u));
}

// ---------------------------------------------------------------- count pass
template <int W>
__device__ __forceinline__ int64_t count_source(const SysView &v, const Src<W> &s, double eps, int lane) {
    const int n = v.norb;
    const int nchunk = (n + 31) >> 5;
    uint32_t singles = 0;
    uint64_t doubles = 0;
    // singles
#pragma unroll
    for (int w = 0; w < W; w++)
        for (uint64_t r = s.d[w]; r; r &= r - 1) {
            const int i = 64 * w + __ffsll((long long)r) - 1;
            const int sg = i & 1;
            for (int c = 0; c < nchunk; c++) {
                const int pa = lane + 32 * c;
                bool keep = false;
                if (pa < n && ((sel2(s.vir, sg) >> pa) & 1ull)) {
                    double acc = single_value<W>(v, s, i, pa);
                    keep = fabs(acc) > eps;
                }
                singles += __popc(__ballot_sync(FULL, keep));
            }
        }
    // doubles: lanes over a, one mask word each
#pragma unroll
    for (int wi = 0; wi < W; wi++)
        for (uint64_t ri = s.d[wi]; ri; ri &= ri - 1) {
            const int i = 64 * wi + __ffsll((long long)ri) - 1;
            const int pi = i >> 1, si = i & 1;
#pragma unroll
            for (int wj = 0; wj < W; wj++) {
                uint64_t rj = s.d[wj];
                if (wj < wi) rj = 0;
                else if (wj == wi) rj &= (i & 63) == 63 ? 0ull : (~0ull << ((i & 63) + 1));
                for (; rj; rj &= rj - 1) {
                    const int j = 64 * wj + __ffsll((long long)rj) - 1;
                    const int pj = j >> 1, sj = j & 1;
                    const int kind = (si == sj) ? 0 : 1;
                    const uint64_t *__restrict__ mrow =
                        v.mask + ((size_t)(kind * n + pi) * n + pj) * v.mrow;
                    for (int c = 0; c < nchunk; c++) {
                        const int pa = lane + 32 * c;
                        if (pa < n && ((sel2(s.vir, si) >> pa) & 1ull))
                            doubles += __popcll(__ldg(mrow + pa) & sel2(s.vir, sj));
                    }
                }
            }
        }
    // warp reduction of the doubles
    unsigned long long d = doubles;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(FULL, d, o);
    return 1 + (int64_t)singles + (int64_t)d;
}


// ---------------------------------------------------------------- staging
// Per-warp double buffer in shared memory holding, for one occupied pair
// (i, j), its integral slab T[pair][a][b] and its screening-mask row, filled by
// bulk asynchronous copies (cp.async.bulk, completion on an mbarrier) one
// pair ahead of the pair being written out.
struct WarpStage {
    double *slab0;     // buffer b at slab0 + b * slab
    uint64_t *mrow0;   // buffer b at mrow0 + b * mrow
    int slab, mrow;
    uint64_t *bar;    // two mbarriers
    uint32_t phase;   // bit b: parity expected next on barrier b
    int next;         // buffer that receives the next first-pair copy
    int32_t *status;  // set to CUSCI_ERR_TIMEOUT if a copy never lands
};

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__host__ __device__ constexpr size_t stage_bytes(int slab, int mrow) {
    return 16 + 2 * ((size_t)slab + (size_t)mrow) * 8;
}

__device__ __forceinline__ void stage_init(WarpStage &st, unsigned char *base, int slab, int mrow,
                                           int lane, int32_t *status) {
    st.bar = reinterpret_cast<uint64_t *>(base);
    st.slab0 = reinterpret_cast<double *>(base + 16);
    st.mrow0 = reinterpret_cast<uint64_t *>(st.slab0 + 2 * slab);
    st.slab = slab;
    st.mrow = mrow;
    st.phase = 0;
    st.next = 0;
    st.status = status;
    if (lane == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(st.bar)) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(st.bar + 1))
                     : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
}

// lane 0 issues the bulk copies of pair q's slab and mask row into buffer b
__device__ __forceinline__ void stage_issue(WarpStage &st, const SysView &v, size_t q, int b,
                                            int lane) {
    __syncwarp();
    if (lane == 0) {
        const uint32_t bs = (uint32_t)v.slab * 8u, bm = (uint32_t)v.mrow * 8u;
        const uint32_t bar = smem_addr(st.bar + b);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                     "r"(bs + bm)
                     : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, "
            "[%3];" ::"r"(smem_addr(st.slab0 + b * st.slab)),
            "l"(v.T + q * v.slab), "r"(bs), "r"(bar)
            : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, "
            "[%3];" ::"r"(smem_addr(st.mrow0 + b * st.mrow)),
            "l"(v.mask + q * v.mrow), "r"(bm), "r"(bar)
            : "memory");
    }
}

// every lane waits (bounded) for buffer b, then flips its expected parity
__device__ __forceinline__ void stage_wait(WarpStage &st, int b) {
    const uint32_t bar = smem_addr(st.bar + b);
    const uint32_t par = (st.phase >> b) & 1u;
    uint32_t done = 0;
    for (int tries = 0; tries < (1 << 22) && !done; tries++) {
        asm volatile(
            "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; "
            "selp.u32 %0, 1, 0, p; }"
            : "=r"(done)
            : "r"(bar), "r"(par)
            : "memory");
    }
    if (!done && st.status) *st.status = CUSCI_ERR_TIMEOUT;
    st.phase ^= 1u << b;
}

// first occupied spin orbital above x (x = -1: the lowest), or -1
template <int W>
__device__ __forceinline__ int next_occ(const uint64_t (&d)[W], int x) {
#pragma unroll
    for (int w = 0; w < W; w++) {
        const int lo = 64 * w;
        if (x >= lo + 63) continue;
        uint64_t r = d[w];
        if (x >= lo) r &= ~0ull << (x - lo + 1);
        if (r) return lo + __ffsll((long long)r) - 1;
    }
    return -1;
}

// position of the n-th (0-based) set bit of x; n < popcount(x) (else some
// position in 0..31 / 0..63, never out of range)
__device__ __forceinline__ int select32(uint32_t x, int n) {
    int pos = 0, c;
    c = __popc(x & 0xFFFFu);
    if (n >= c) { n -= c; pos += 16; x >>= 16; }
    c = __popc(x & 0xFFu);
    if (n >= c) { n -= c; pos += 8; x >>= 8; }
    c = __popc(x & 0xFu);
    if (n >= c) { n -= c; pos += 4; x >>= 4; }
    c = __popc(x & 0x3u);
    if (n >= c) { n -= c; pos += 2; x >>= 2; }
    if (n >= (int)(x & 1u)) pos += 1;
    return pos;
}

__device__ __forceinline__ int select64(uint64_t x, int n) {
    const uint32_t lo = (uint32_t)x;
    const int cl = __popc(lo);
    return n < cl ? select32(lo, n) : 32 + select32((uint32_t)(x >> 32), n - cl);
}

// slab index of the occupied pair (i < j): kind 0 same spin, 1 opposite
__device__ __forceinline__ size_t pair_index(int n, int i, int j) {
    const int kind = ((i ^ j) & 1) ? 1 : 0;
    return (size_t)(kind * n + (i >> 1)) * n + (j >> 1);
}

// Visits every kept entry of the coupled set of source s in canonical order.
// emit(t, h, rank) is called by the lane that owns the entry: t is the target
// determinant, h the signed FP64 element, rank its position in the source's
// list (0 = diagonal).  emit.pair_possible(tij, si, sj) / emit.row_possible(
// tija, sj) may rule out every double of an occupied pair (tij: source with i
// and j removed) or of a row (tija: also a added); emitters that need exact
// positions must return true.  The call is warp-collective (all 32 lanes, uniform
// control flow); returns |C_s|.
template <int W, class Emit>
__device__ __forceinline__ int64_t visit_source(const SysView &v, const Src<W> &s, double eps,
                                                int lane, Emit &emit, WarpStage *stg = nullptr) {
    const int n = v.norb;
    const int nchunk = (n + 31) >> 5;
    int64_t pos = 0;
    // prefetch the first occupied pair while the diagonal and singles run
    const int i0 = next_occ<W>(s.d, -1);
    const int j0 = i0 >= 0 ? next_occ<W>(s.d, i0) : -1;
    if (stg && j0 >= 0) stage_issue(*stg, v, pair_index(n, i0, j0), stg->next, lane);
    // 1. diagonal
    {
        double hd = diagonal_value<W>(v, s);
        if (lane == 0) emit(s.d, hd, pos);
        pos += 1;
    }
    // 2. singles
#pragma unroll
    for (int w = 0; w < W; w++)
        for (uint64_t r = s.d[w]; r; r &= r - 1) {
            const int i = 64 * w + __ffsll((long long)r) - 1;
            const int sg = i & 1;
            const uint32_t ni = par_bit(s.par, i);
            for (int c = 0; c < nchunk; c++) {
                const int pa = lane + 32 * c;
                bool keep = false;
                double acc = 0.0;
                if (pa < n && ((sel2(s.vir, sg) >> pa) & 1ull)) {
                    acc = single_value<W>(v, s, i, pa);
                    keep = fabs(acc) > eps;
                }
                const uint32_t b = __ballot_sync(FULL, keep);
                if (keep) {
                    const int a = 2 * pa + sg;
                    const uint32_t odd = ni ^ par_bit(s.par, a) ^ (uint32_t)(i < a);
                    uint64_t t[W];
#pragma unroll
                    for (int q = 0; q < W; q++) t[q] = s.d[q];
                    flip_bit<W>(t, i);
                    flip_bit<W>(t, a);
                    emit(t, flip_sign(acc, odd), pos + lanes_below(b, lane));
                }
                pos += __popc(b);
            }
        }
    // 3. doubles, one occupied pair (i < j) at a time in canonical order.
    // Per pair the surviving (a, b) are expanded across the warp: lanes first
    // take rows (virtual a of i's spin, ascending, 32 per group) and prefix-sum
    // their survivor counts; then every lane takes one output slot k, finds its
    // row by a search over the lanes' prefix sums and its b as the
    // (k - prefix)-th set bit of the row's mask.  All lanes stay busy whatever
    // the mask density.
    int cur = stg ? stg->next : 0;
    for (int i = i0, j = j0; j >= 0;) {
        int ni = i, nj = next_occ<W>(s.d, j);
        if (nj < 0) {
            ni = next_occ<W>(s.d, i);
            nj = ni >= 0 ? next_occ<W>(s.d, ni) : -1;
        }
        const int si = i & 1, sj = j & 1;
        const size_t q = pair_index(n, i, j);
        const double *__restrict__ slab;
        const uint64_t *__restrict__ mrow;
        if (stg) {
            if (nj >= 0) stage_issue(*stg, v, pair_index(n, ni, nj), cur ^ 1, lane);
            stage_wait(*stg, cur);
            slab = stg->slab0 + cur * stg->slab;
            mrow = stg->mrow0 + cur * stg->mrow;
        } else {
            slab = v.T + q * v.slab;
            mrow = v.mask + q * v.mrow;
        }
        const uint32_t nij = par_bit(s.par, i) ^ par_bit(s.par, j) ^ 1u;
        uint64_t tij[W];
#pragma unroll
        for (int w = 0; w < W; w++) tij[w] = s.d[w];
        flip_bit<W>(tij, i);
        flip_bit<W>(tij, j);
        const uint64_t virj = sel2(s.vir, sj);
        const uint64_t parj = sel2(s.par, sj);
        // an emitter may rule out a whole pair (all its targets lie outside the
        // set it looks targets up in); positions then stop counting that pair,
        // which only emitters that ignore positions may do
        const bool pair_live = emit.pair_possible(tij, si, sj);
        for (uint64_t vs = pair_live ? sel2(s.vir, si) : 0ull; vs;) {
            // row of this lane: the lane-th remaining virtual a
            const int rows = __popcll(vs) < 32 ? __popcll(vs) : 32;
            int pa = -1;
            uint64_t m = 0;
            if (lane < rows) {
                pa = select64(vs, lane);
                m = (stg ? mrow[pa] : __ldg(mrow + pa)) & virj;
                if (m) {
                    uint64_t tija[W];
#pragma unroll
                    for (int w = 0; w < W; w++) tija[w] = tij[w];
                    flip_bit<W>(tija, 2 * pa + si);
                    if (!emit.row_possible(tija, sj)) m = 0;
                }
            }
            const uint32_t cnt = (uint32_t)__popcll(m);
            uint32_t incl = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(FULL, incl, o);
                if (lane >= o) incl += y;
            }
            const uint32_t excl = incl - cnt;
            const uint32_t total = __shfl_sync(FULL, incl, 31);
            const int a_l = 2 * pa + si;
            const uint32_t cija_l =
                nij ^ (pa >= 0 ? par_bit(s.par, a_l) : 0u) ^ (uint32_t)(i < a_l) ^ (uint32_t)(j < a_l);
            for (uint32_t k0 = 0; k0 < total; k0 += 32) {
                const uint32_t k = k0 + lane;
                int r = 0;
#pragma unroll
                for (int step = 16; step >= 1; step >>= 1) {
                    const int cand = r + step;
                    const uint32_t e = __shfl_sync(FULL, excl, cand & 31);
                    if (cand < rows && e <= k) r = cand;
                }
                const uint64_t mr = __shfl_sync(FULL, m, r);
                const uint32_t er = __shfl_sync(FULL, excl, r);
                const int par_r = __shfl_sync(FULL, pa, r);
                const uint32_t cr = __shfl_sync(FULL, cija_l, r);
                if (k < total) {
                    const int pb = select64(mr, (int)(k - er));
                    const int a = 2 * par_r + si, b = 2 * pb + sj;
                    const uint32_t odd = cr ^ (uint32_t)((parj >> pb) & 1ull) ^ (uint32_t)(i < b) ^
                                         (uint32_t)(j < b) ^ (uint32_t)(b < a);
                    uint64_t t[W];
#pragma unroll
                    for (int w = 0; w < W; w++) t[w] = tij[w];
                    flip_bit<W>(t, a);
                    flip_bit<W>(t, b);
                    const double val = stg ? slab[par_r * n + pb] : __ldg(slab + par_r * n + pb);
                    emit(t, flip_sign(val, odd), pos + k);
                }
            }
            pos += total;
            // drop the rows just handled
            if (rows >= __popcll(vs)) {
                vs = 0;
            } else {
                const int last = select64(vs, rows - 1);
                vs &= ~0ull << (last + 1);
            }
        }
        if (stg) {
            __syncwarp();
            cur ^= 1;
        }
        i = ni;
        j = nj;
    }
    if (stg) stg->next = cur;
    return pos;
}

}  // namespace enumr
}  // namespace cusci
