// LSD radix-sort building blocks (8-bit digits, reduce-then-scan over a
// persistent grid) shared by the de-duplication paths.
#pragma once

#include "cusci_internal.cuh"

namespace cusci {
namespace radix {

constexpr int RT = 256;          // threads per CTA
constexpr int RI = 8;            // keys per thread per tile
constexpr int RTILE = RT * RI;   // 2048
constexpr int RBITS = 8;
constexpr int RADIX = 1 << RBITS;
constexpr int RWARPS = RT / 32;
constexpr int BINOM_K = 65;      // binom[m][k], m < 128, k <= 64
constexpr unsigned FULL = 0xffffffffu;


template <int KW>
struct Key {
    uint64_t w[KW];
};

template <int KW>
__device__ __forceinline__ uint32_t digit_of(const Key<KW> &k, int shift) {
    if (KW == 1) return (uint32_t)((k.w[0] >> shift) & (RADIX - 1));
    // KW == 2; the word is chosen by a select, not an index, so that keys held
    // in registers are not moved to local memory
    const int word = shift >> 6, sh = shift & 63;
    uint64_t lo = (word == 0 ? k.w[0] : k.w[KW - 1]) >> sh;
    if (sh > 64 - RBITS && word + 1 < KW) lo |= k.w[KW - 1] << (64 - sh);
    return (uint32_t)(lo & (RADIX - 1));
}

template <int KW>
__device__ __forceinline__ bool key_eq(const Key<KW> &a, const Key<KW> &b) {
#pragma unroll
    for (int q = 0; q < KW; q++)
        if (a.w[q] != b.w[q]) return false;
    return true;
}

// ------------------------------------------------------------------ radix pass
template <int KW>
__global__ void __launch_bounds__(RT)
    upsweep(const Key<KW> *__restrict__ keys, int64_t total, int shift, int64_t per_cta,
            uint32_t *__restrict__ hist) {
    __shared__ uint32_t h[RADIX];
    for (int d = threadIdx.x; d < RADIX; d += RT) h[d] = 0;
    __syncthreads();
    const int64_t beg = (int64_t)blockIdx.x * per_cta;
    int64_t end = beg + per_cta;
    if (end > total) end = total;
    for (int64_t k = beg + threadIdx.x; k < end; k += RT) atomicAdd(&h[digit_of<KW>(keys[k], shift)], 1u);
    __syncthreads();
    for (int d = threadIdx.x; d < RADIX; d += RT) hist[(int64_t)d * gridDim.x + blockIdx.x] = h[d];
}

template <int KW>
struct alignas(16) DownSmem {
    Key<KW> keys[RTILE];
    uint32_t idx[RTILE];
    uint32_t warp_cnt[RWARPS][RADIX];
    uint32_t tile_cnt[RADIX];
    uint32_t tile_start[RADIX];
    int64_t running[RADIX];
};

template <int KW>
__global__ void __launch_bounds__(RT)
    downsweep(const Key<KW> *__restrict__ kin, const uint32_t *__restrict__ iin,
              Key<KW> *__restrict__ kout, uint32_t *__restrict__ iout, int64_t total, int shift,
              int64_t per_cta, const int64_t *__restrict__ base) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    DownSmem<KW> &S = *reinterpret_cast<DownSmem<KW> *>(smem_raw);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int d = threadIdx.x; d < RADIX; d += RT)
        S.running[d] = base[(int64_t)d * gridDim.x + blockIdx.x];
    const int64_t cbeg = (int64_t)blockIdx.x * per_cta;
    int64_t cend = cbeg + per_cta;
    if (cend > total) cend = total;

    for (int64_t t0 = cbeg; t0 < cend; t0 += RTILE) {
        const int64_t tn64 = cend - t0;
        const int tn = tn64 < RTILE ? (int)tn64 : RTILE;
        for (int q = threadIdx.x; q < RWARPS * RADIX; q += RT) (&S.warp_cnt[0][0])[q] = 0;
        __syncthreads();
        // each warp ranks its contiguous sub-tile of RI*32 keys, 32 per round
        Key<KW> k[RI];
        uint32_t id[RI], dg[RI], rk[RI];
#pragma unroll
        for (int r = 0; r < RI; r++) {
            const int e = wid * (RI * 32) + r * 32 + lane;
            const bool valid = e < tn;
            if (valid) {
                k[r] = kin[t0 + e];
                id[r] = iin[t0 + e];
                dg[r] = digit_of<KW>(k[r], shift);
            } else {
                dg[r] = RADIX;  // sentinel, never stored
            }
            const unsigned peers = __match_any_sync(FULL, dg[r]);
            const int below = __popc(peers & ((1u << lane) - 1u));
            uint32_t prev = 0;
            if (valid) prev = S.warp_cnt[wid][dg[r]];
            rk[r] = prev + below;
            __syncwarp();
            if (valid && below == 0) S.warp_cnt[wid][dg[r]] = prev + __popc(peers);
            __syncwarp();
        }
        __syncthreads();
        // per digit: exclusive prefix over warps, tile totals
        for (int d = threadIdx.x; d < RADIX; d += RT) {
            uint32_t s = 0;
#pragma unroll
            for (int w = 0; w < RWARPS; w++) {
                uint32_t c = S.warp_cnt[w][d];
                S.warp_cnt[w][d] = s;
                s += c;
            }
            S.tile_cnt[d] = s;
        }
        __syncthreads();
        // exclusive scan of tile_cnt over digits (one warp)
        if (wid == 0) {
            uint32_t carry = 0;
            for (int d0 = 0; d0 < RADIX; d0 += 32) {
                uint32_t x = S.tile_cnt[d0 + lane], inc = x;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    uint32_t y = __shfl_up_sync(FULL, inc, o);
                    if (lane >= o) inc += y;
                }
                S.tile_start[d0 + lane] = carry + inc - x;
                carry += __shfl_sync(FULL, inc, 31);
            }
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < RI; r++) {
            if (dg[r] < RADIX) {
                const uint32_t p = S.tile_start[dg[r]] + S.warp_cnt[wid][dg[r]] + rk[r];
                S.keys[p] = k[r];
                S.idx[p] = id[r];
            }
        }
        __syncthreads();
        for (int p = threadIdx.x; p < tn; p += RT) {
            const Key<KW> kk = S.keys[p];
            const uint32_t d = digit_of<KW>(kk, shift);
            const int64_t dst = S.running[d] + (p - (int64_t)S.tile_start[d]);
            kout[dst] = kk;
            iout[dst] = S.idx[p];
        }
        __syncthreads();
        for (int d = threadIdx.x; d < RADIX; d += RT) S.running[d] += S.tile_cnt[d];
        __syncthreads();
    }
}


}  // namespace radix
}  // namespace cusci
