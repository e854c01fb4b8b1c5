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

__device__ __forceinline__ uint32_t par_bit(const uint64_t par[2], int so) {
    return (uint32_t)((par[so & 1] >> (so >> 1)) & 1ull);
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
__device__ int64_t count_source(const SysView &v, const Src<W> &s, double eps, int lane) {
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
                if (pa < n && ((s.vir[sg] >> pa) & 1ull)) {
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
                        v.mask + ((size_t)(kind * n + pi) * n + pj) * n;
                    for (int c = 0; c < nchunk; c++) {
                        const int pa = lane + 32 * c;
                        if (pa < n && ((s.vir[si] >> pa) & 1ull))
                            doubles += __popcll(__ldg(mrow + pa) & s.vir[sj]);
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


// Visits every kept entry of the coupled set of source s in canonical order.
// emit(t, h, rank) is called by the lane that owns the entry: t is the target
// determinant, h the signed FP64 element, rank its position in the source's
// list (0 = diagonal).  The call is warp-collective (all 32 lanes, uniform
// control flow); returns |C_s|.
template <int W, class Emit>
__device__ __forceinline__ int64_t visit_source(const SysView &v, const Src<W> &s, double eps,
                                                int lane, Emit &emit) {
    const int n = v.norb;
    const int nchunk = (n + 31) >> 5;
    int64_t pos = 0;
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
                if (pa < n && ((s.vir[sg] >> pa) & 1ull)) {
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
    // 3. doubles
#pragma unroll
    for (int wi = 0; wi < W; wi++)
        for (uint64_t ri = s.d[wi]; ri; ri &= ri - 1) {
            const int i = 64 * wi + __ffsll((long long)ri) - 1;
            const int pi = i >> 1, si = i & 1;
            const uint32_t ni = par_bit(s.par, i);
#pragma unroll
            for (int wj = 0; wj < W; wj++) {
                uint64_t rj = s.d[wj];
                if (wj < wi) rj = 0;
                else if (wj == wi) rj &= (i & 63) == 63 ? 0ull : (~0ull << ((i & 63) + 1));
                for (; rj; rj &= rj - 1) {
                    const int j = 64 * wj + __ffsll((long long)rj) - 1;
                    const int pj = j >> 1, sj = j & 1;
                    const int kind = (si == sj) ? 0 : 1;
                    const size_t row0 = ((size_t)(kind * n + pi) * n + pj) * n;
                    const uint64_t *__restrict__ mrow = v.mask + row0;
                    const uint32_t nij = ni ^ par_bit(s.par, j) ^ 1u;
                    uint64_t tij[W];
#pragma unroll
                    for (int q = 0; q < W; q++) tij[q] = s.d[q];
                    flip_bit<W>(tij, i);
                    flip_bit<W>(tij, j);
                    for (uint64_t ra = s.vir[si]; ra; ra &= ra - 1) {
                        const int pa = __ffsll((long long)ra) - 1;
                        const uint64_t m = __ldg(mrow + pa) & s.vir[sj];
                        if (m == 0) continue;
                        const int a = 2 * pa + si;
                        const uint32_t cija =
                            nij ^ par_bit(s.par, a) ^ (uint32_t)(i < a) ^ (uint32_t)(j < a);
                        const double *__restrict__ trow = v.T + (row0 + pa) * n;
                        for (int c = 0; c < nchunk; c++) {
                            const int pb = lane + 32 * c;
                            if (pb < n && ((m >> pb) & 1ull)) {
                                const int b = 2 * pb + sj;
                                const int64_t p =
                                    pos + __popcll(m & ((pb == 0) ? 0ull : (~0ull >> (64 - pb))));
                                const uint32_t odd = cija ^ par_bit(s.par, b) ^ (uint32_t)(i < b) ^
                                                     (uint32_t)(j < b) ^ (uint32_t)(b < a);
                                uint64_t t[W];
#pragma unroll
                                for (int q = 0; q < W; q++) t[q] = tij[q];
                                flip_bit<W>(t, a);
                                flip_bit<W>(t, b);
                                emit(t, flip_sign(__ldg(trow + pb), odd), p);
                            }
                        }
                        pos += __popcll(m);
                    }
                }
            }
        }
    return pos;
}

}  // namespace enumr
}  // namespace cusci
