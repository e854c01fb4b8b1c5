// Streaming generation + de-duplication in mini-batches out of a caller-owned
// device pool (the GPU memory-centric execution of Sec. 4.3, Stage 1).
//
//  * all sources are counted once; the host cuts them into mini-batches whose
//    coupled lists fit one half of the pool's batch region, so peak device
//    memory depends on the pool size only (Sec. 4.3.2);
//  * batch k is filled into buffer k % 2 while batch k-1 is copied to the
//    caller's pinned host sinks on a side stream (double buffering, Sec. 4.3.3);
//    cold data -- the original coupled set -- lives on the host, as in the
//    paper's Stage 1 offload;
//  * every batch's targets go into one device-wide open-addressing hash set
//    (the in-batch de-duplication spanning all batches); slots are claimed
//    with atomicCAS on the first key word, the second word is published right
//    after, and a reader that meets a claimed slot with an equal first word
//    waits (bounded) for the second;
//  * finally the distinct keys are compacted out of the hash set and sorted
//    with the library's de-duplication into the caller's output.

#include <chrono>
#include <stdlib.h>
#include <string.h>

#include "enumerate.cuh"

namespace cusci {
cusci_status exclusive_scan_i64(const int64_t *in, int64_t n, int64_t *out, int64_t *ws,
                                cudaStream_t st);
int64_t scan_tiles(int64_t n);

namespace {

constexpr uint64_t EMPTY = ~0ull;
constexpr int HT = 256;
// polls of a slot's second key word before a two-word insert gives up
// (another thread has claimed the slot's first word and writes the second
// right after)
constexpr int SPIN_LIMIT = 1 << 20;

__device__ __forceinline__ uint64_t mix64s(uint64_t x) {
    x ^= x >> 31;
    x *= 0x7fb5d329728ea185ull;
    x ^= x >> 27;
    x *= 0x81dadef4bc2dd44dull;
    x ^= x >> 33;
    return x;
}

template <int W>
__global__ void __launch_bounds__(HT)
    hash_insert(const uint64_t *__restrict__ keys, int64_t n, uint64_t *__restrict__ tab,
                uint64_t mask, unsigned long long *__restrict__ n_new,
                int32_t *__restrict__ status, int spin_limit) {
    unsigned long long mine = 0;
    for (int64_t k = blockIdx.x * (int64_t)HT + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * HT) {
        uint64_t x[W];
#pragma unroll
        for (int w = 0; w < W; w++) x[w] = keys[k * W + w];
        uint64_t h = mix64s(x[0] ^ (W == 2 ? mix64s(x[W - 1] + 0x9e3779b97f4a7c15ull) : 0ull));
        h &= mask;
        bool done = false;
        for (uint64_t probe = 0; probe <= mask && !done; probe++) {
            uint64_t *slot = tab + h * W;
            const unsigned long long old =
                atomicCAS((unsigned long long *)slot, (unsigned long long)EMPTY,
                          (unsigned long long)x[0]);
            if (old == EMPTY) {
                if (W == 2) *(volatile uint64_t *)(slot + 1) = x[W - 1];
                mine++;
                done = true;
            } else if (old == x[0]) {
                if (W == 1) {
                    done = true;
                } else {
                    uint64_t second = EMPTY;
                    for (int spin = 0; spin < spin_limit; spin++) {
                        second = *(volatile uint64_t *)(slot + 1);
                        if (second != EMPTY) break;
                    }
                    if (second == EMPTY) {
                        if (status) *status = CUSCI_ERR_TIMEOUT;
                        done = true;
                    } else if (second == x[W - 1]) {
                        done = true;
                    }
                }
            }
            h = (h + 1) & mask;
        }
        if (!done && status) *status = CUSCI_ERR_OVERFLOW;  // table full
    }
    // block total of new keys, one atomic per block
    __shared__ unsigned long long red[HT / 32];
    for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mine;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long s = 0;
        for (int w = 0; w < HT / 32; w++) s += red[w];
        if (s) atomicAdd(n_new, s);
    }
}

// block-aggregated compaction of the occupied slots (one atomic per block)
template <int W>
__global__ void __launch_bounds__(HT)
    hash_compact(const uint64_t *__restrict__ tab, uint64_t cap, uint64_t *__restrict__ out,
                 unsigned long long *__restrict__ cursor, int64_t out_cap,
                 int32_t *__restrict__ status) {
    __shared__ uint32_t wcount[HT / 32];
    __shared__ unsigned long long base;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const uint64_t stride = (uint64_t)gridDim.x * HT;
    for (uint64_t k0 = blockIdx.x * (uint64_t)HT; k0 < cap; k0 += stride) {
        const uint64_t k = k0 + threadIdx.x;
        const bool full = k < cap && tab[k * W] != EMPTY;
        const unsigned bal = __ballot_sync(0xffffffffu, full);
        if (lane == 0) wcount[wid] = __popc(bal);
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t s = 0;
            for (int w = 0; w < HT / 32; w++) {
                const uint32_t c = wcount[w];
                wcount[w] = s;
                s += c;
            }
            base = s ? atomicAdd(cursor, (unsigned long long)s) : 0ull;
        }
        __syncthreads();
        if (full) {
            const unsigned long long at = base + wcount[wid] + __popc(bal & ((1u << lane) - 1u));
            if ((int64_t)at < out_cap) {
#pragma unroll
                for (int w = 0; w < W; w++) out[at * W + w] = tab[k * W + w];
            } else if (status) {
                *status = CUSCI_ERR_OVERFLOW;
            }
        }
        __syncthreads();
    }
}

__global__ void rel_offsets(const int64_t *__restrict__ abs_off, int64_t n,
                            int64_t *__restrict__ rel) {
    const int64_t base = abs_off[0];
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x)
        rel[k] = abs_off[k] - base;
}

size_t al(size_t x) { return (x + 255) & ~(size_t)255; }

// power of two holding unique_capacity keys at a load of at most 3/4
uint64_t table_slots(int64_t unique_capacity) {
    uint64_t c = 1024;
    while (c < (uint64_t)unique_capacity + (uint64_t)unique_capacity / 3) c <<= 1;
    return c;
}

// Pool layout: [per-source arrays][control words][X], X reused by the two
// phases.  Phase 1 (batches): the hash table at X, the two batch buffers
// after it.  Phase 2 (final sort): the inverse and the sort workspace ("tail")
// at X over the dead table, the compacted distinct keys after max(table, tail)
// (never inside the table, which the compaction reads).
size_t inv_bytes(int64_t unique_capacity) {
    return unique_capacity < ((int64_t)1 << 31) ? 4 : 8;
}

size_t sort_tail(int64_t unique_capacity, size_t ws) {
    return al((size_t)unique_capacity * inv_bytes(unique_capacity)) + al(ws);
}

}  // namespace
}  // namespace cusci

using namespace cusci;

extern "C" cusci_status cusci_stream_pool_bytes(const cusci_system *sys, int64_t n_sources,
                                                int64_t batch_entries, int64_t unique_capacity,
                                                size_t *bytes) {
    if (!sys || !bytes || n_sources < 0 || batch_entries < 1 || unique_capacity < 1)
        return fail(CUSCI_ERR_INVALID, "cusci_stream_pool_bytes: bad argument");
    const int W = sys->W;
    const size_t tab = al(table_slots(unique_capacity) * 8 * W);
    const size_t per_src = al((size_t)(n_sources + 1) * 8) * 3 + al((size_t)n_sources * 8 * W);
    const size_t bat = 2 * (al((size_t)batch_entries * 8 * W) + al((size_t)batch_entries * 8));
    size_t ws = 0;
    cusci_dedup_workspace(unique_capacity, W, 2 * sys->norb, sys->n_alpha + sys->n_beta, &ws);
    const size_t tail = sort_tail(unique_capacity, ws);
    const size_t phase1 = tab + bat;
    const size_t phase2 = (tail > tab ? tail : tab) + al((size_t)unique_capacity * 8 * W);
    *bytes = per_src + al(4096) + (phase1 > phase2 ? phase1 : phase2);
    return CUSCI_OK;
}

extern "C" cusci_status cusci_stream_gen_dedup(
    const cusci_system *sys, const uint64_t *h_dets, int64_t n, double eps, void *d_pool,
    size_t pool_bytes, int64_t batch_entries, int64_t *h_offsets, uint64_t *h_out_dets,
    double *h_out_h, int64_t host_capacity, uint64_t *d_unique, int64_t unique_capacity,
    int64_t *h_n_unique, int64_t *h_stats, void *stream) {
    if (!sys || n < 0 || !h_dets || !d_pool || !h_offsets || !d_unique || !h_n_unique ||
        batch_entries < 1 || unique_capacity < 1)
        return fail(CUSCI_ERR_INVALID, "cusci_stream_gen_dedup: bad argument");
    if (eps != eps) return fail(CUSCI_ERR_INVALID, "cusci_stream_gen_dedup: eps is NaN");
    const int W = sys->W;
    const int N1 = sys->n_alpha + sys->n_beta;
    if (N1 >= 64)
        return fail(CUSCI_ERR_UNSUPPORTED, "cusci_stream_gen_dedup: needs fewer than 64 electrons");
    size_t need = 0;
    cusci_status rc = cusci_stream_pool_bytes(sys, n, batch_entries, unique_capacity, &need);
    if (rc != CUSCI_OK) return rc;
    if (pool_bytes < need)
        return fail(CUSCI_ERR_OOM, "cusci_stream_gen_dedup: pool %zu < %zu bytes", pool_bytes, need);
    if ((uintptr_t)d_pool & 255u) return fail(CUSCI_ERR_INVALID, "stream: pool not 256-aligned");
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e;
    const auto t_start = std::chrono::steady_clock::now();

    // carve the pool
    unsigned char *p = (unsigned char *)d_pool;
    const uint64_t slots = table_slots(unique_capacity);
    const size_t tab_bytes = al(slots * 8 * W);
    int64_t *d_counts = (int64_t *)p; p += al((size_t)(n + 1) * 8);
    int64_t *d_off = (int64_t *)p; p += al((size_t)(n + 1) * 8);
    int64_t *d_boff = (int64_t *)p; p += al((size_t)(n + 1) * 8);
    uint64_t *d_src = (uint64_t *)p; p += al((size_t)n * 8 * W);
    unsigned char *phase = p;
    unsigned long long *d_ctr = (unsigned long long *)phase;   // [0] new keys, [1] compaction
    int32_t *d_status = (int32_t *)(phase + 64);
    unsigned char *X = phase + al(4096);
    uint64_t *tab = (uint64_t *)X;
    unsigned char *bat = X + tab_bytes;
    uint64_t *bd[2];
    double *bh[2];
    bd[0] = (uint64_t *)bat; bat += al((size_t)batch_entries * 8 * W);
    bh[0] = (double *)bat; bat += al((size_t)batch_entries * 8);
    bd[1] = (uint64_t *)bat; bat += al((size_t)batch_entries * 8 * W);
    bh[1] = (double *)bat; bat += al((size_t)batch_entries * 8);
    const size_t peak1 = (size_t)(bat - (unsigned char *)d_pool);

    e = cudaMemsetAsync(tab, 0xff, slots * 8 * W, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(phase, 0, 4096, st);
    if (e == cudaSuccess && n > 0)
        e = cudaMemcpyAsync(d_src, h_dets, (size_t)n * 8 * W, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "stream: setup");

    // counts of every source, read back to plan the batches
    rc = cusci_count_coupled(sys, d_src, n, eps, d_counts, stream);
    if (rc != CUSCI_OK) return rc;
    int64_t *h_counts = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * 8);
    if (!h_counts) return fail(CUSCI_ERR_OOM, "stream: host allocation");
    if (n > 0) e = cudaMemcpyAsync(h_counts, d_counts, (size_t)n * 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        free(h_counts);
        return cuda_fail(e, "stream: counts");
    }
    h_offsets[0] = 0;
    for (int64_t k = 0; k < n; k++) {
        if (h_counts[k] > batch_entries) {
            free(h_counts);
            return fail(CUSCI_ERR_OOM, "stream: source %lld has %lld entries > batch capacity %lld",
                        (long long)k, (long long)h_counts[k], (long long)batch_entries);
        }
        h_offsets[k + 1] = h_offsets[k] + h_counts[k];
    }
    free(h_counts);
    const int64_t total = h_offsets[n];
    const bool offload = h_out_dets && h_out_h;
    if (offload && total > host_capacity)
        return fail(CUSCI_ERR_OOM, "stream: host sinks hold %lld entries, need %lld",
                    (long long)host_capacity, (long long)total);

    // all offsets to the device once (batches take batch-relative views of them)
    e = cudaMemcpyAsync(d_boff, h_offsets, (size_t)(n + 1) * 8, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "stream: offsets");
    cudaStream_t cp;
    e = cudaStreamCreateWithFlags(&cp, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(e, "stream: copy stream");
    cudaEvent_t filled[2], copied[2];
    bool have_copy[2] = {false, false};
    for (int b = 0; b < 2; b++) {
        cudaEventCreateWithFlags(&filled[b], cudaEventDisableTiming);
        cudaEventCreateWithFlags(&copied[b], cudaEventDisableTiming);
    }
    int64_t nbatch = 0;
    rc = CUSCI_OK;
    for (int64_t s0 = 0; s0 < n && rc == CUSCI_OK;) {
        // greedy batch of whole sources
        int64_t s1 = s0;
        while (s1 < n && h_offsets[s1 + 1] - h_offsets[s0] <= batch_entries) s1++;
        const int buf = (int)(nbatch & 1);
        const int64_t be = h_offsets[s1] - h_offsets[s0];
        // the buffer's previous copy must have left before it is overwritten
        if (have_copy[buf]) {
            e = cudaStreamWaitEvent(st, copied[buf], 0);
            if (e != cudaSuccess) { rc = cuda_fail(e, "stream: wait"); break; }
        }
        // batch-relative offsets from the device copy of all offsets
        rel_offsets<<<(int)((s1 - s0 + 256) / 256), 256, 0, st>>>(d_boff + s0, s1 - s0 + 1, d_off);
        note_launches(1);
        rc = cusci_gen_coupled(sys, d_src + s0 * W, s1 - s0, eps, d_off, bd[buf], bh[buf],
                               d_status, stream);
        if (rc != CUSCI_OK) break;
        int blocks = (int)((be + HT - 1) / HT);
        if (blocks > sm_count() * 8) blocks = sm_count() * 8;
        if (blocks < 1) blocks = 1;
        if (W == 1)
            hash_insert<1><<<blocks, HT, 0, st>>>(bd[buf], be, tab, slots - 1, d_ctr, d_status,
                                                  SPIN_LIMIT);
        else
            hash_insert<2><<<blocks, HT, 0, st>>>(bd[buf], be, tab, slots - 1, d_ctr, d_status,
                                                  SPIN_LIMIT);
        e = cudaGetLastError();
        if (e != cudaSuccess) { rc = cuda_fail(e, "stream: hash insert"); break; }
        note_launches(1);
        if (offload && be > 0) {
            e = cudaEventRecord(filled[buf], st);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(cp, filled[buf], 0);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(h_out_dets + h_offsets[s0] * W, bd[buf], (size_t)be * 8 * W,
                                    cudaMemcpyDeviceToHost, cp);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(h_out_h + h_offsets[s0], bh[buf], (size_t)be * 8,
                                    cudaMemcpyDeviceToHost, cp);
            if (e == cudaSuccess) e = cudaEventRecord(copied[buf], cp);
            if (e != cudaSuccess) { rc = cuda_fail(e, "stream: offload"); break; }
            have_copy[buf] = true;
        }
        nbatch++;
        s0 = s1;
    }
    // drain the copies
    cudaError_t e2 = cudaStreamSynchronize(cp);
    if (rc == CUSCI_OK && e2 != cudaSuccess) rc = cuda_fail(e2, "stream: drain");
    for (int b = 0; b < 2; b++) {
        cudaEventDestroy(filled[b]);
        cudaEventDestroy(copied[b]);
    }
    cudaStreamDestroy(cp);
    if (rc != CUSCI_OK) return rc;

    // distinct keys out of the hash set, then sorted into d_unique
    unsigned long long h_new = 0;
    int32_t h_status = 0;
    e = cudaMemcpyAsync(&h_new, d_ctr, 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h_status, d_status, 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "stream: readback");
    if (h_status != 0)
        return fail((cusci_status)h_status, "stream: device reported status %d (table too small "
                    "or inconsistent counts)", h_status);
    if ((int64_t)h_new > unique_capacity)
        return fail(CUSCI_ERR_OVERFLOW, "stream: %llu distinct keys > capacity %lld", h_new,
                    (long long)unique_capacity);
    const int64_t nu = (int64_t)h_new;
    const auto t_batches = std::chrono::steady_clock::now();
    // phase 2: inverse and sort workspace over the table, compacted keys after
    size_t ws = 0;
    cusci_dedup_workspace(nu > 0 ? nu : 1, W, 2 * sys->norb, N1, &ws);
    const size_t tail = sort_tail(unique_capacity, ws);
    void *inv = X;
    void *dws = X + al((size_t)unique_capacity * inv_bytes(unique_capacity));
    uint64_t *raw = (uint64_t *)(X + (tail > tab_bytes ? tail : tab_bytes));
    const unsigned char *q = (const unsigned char *)raw + al((size_t)unique_capacity * 8 * W);
    const size_t peak2 = (size_t)(q - (unsigned char *)d_pool);
    if (peak2 > pool_bytes) return fail(CUSCI_ERR_OOM, "stream: pool too small for the final sort");
    int cb = (int)((slots + HT - 1) / HT);
    if (cb > sm_count() * 8) cb = sm_count() * 8;
    if (W == 1)
        hash_compact<1><<<cb, HT, 0, st>>>(tab, slots, raw, d_ctr + 1, unique_capacity, d_status);
    else
        hash_compact<2><<<cb, HT, 0, st>>>(tab, slots, raw, d_ctr + 1, unique_capacity, d_status);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "stream: compaction");
    note_launches(1);
    int64_t nu2 = 0;
    rc = cusci_dedup(raw, nu, W, 2 * sys->norb, N1, dws, ws, d_unique, inv,
                     nu < ((int64_t)1 << 31) ? 4 : 8, d_counts + n, &nu2, d_status, stream);
    if (rc != CUSCI_OK) return rc;
    if (nu2 != nu) return fail(CUSCI_ERR_INVALID, "stream: sort of distinct keys lost keys");
    *h_n_unique = nu;
    if (h_stats) {
        h_stats[0] = total;
        h_stats[1] = nbatch;
        h_stats[2] = (int64_t)(peak1 > peak2 ? peak1 : peak2);
        h_stats[3] = offload ? total * (8 * W + 8) : 0;
        const auto t_end = std::chrono::steady_clock::now();
        h_stats[4] = std::chrono::duration_cast<std::chrono::microseconds>(t_batches - t_start).count();
        h_stats[5] = std::chrono::duration_cast<std::chrono::microseconds>(t_end - t_batches).count();
    }
    return CUSCI_OK;
}

extern "C" cusci_status cusci_hash_insert_probe(const uint64_t *d_keys, int64_t n, int W,
                                                uint64_t *d_table, int64_t slots, int spin_limit,
                                                unsigned long long *d_n_new, int32_t *d_status,
                                                void *stream) {
    if (n < 0 || (W != 1 && W != 2) || slots < 1 || (slots & (slots - 1)) || spin_limit < 0)
        return fail(CUSCI_ERR_INVALID, "cusci_hash_insert_probe: bad argument");
    if (n == 0) return CUSCI_OK;
    if (!d_keys || !d_table || !d_n_new)
        return fail(CUSCI_ERR_INVALID, "cusci_hash_insert_probe: NULL buffer");
    int blocks = (int)((n + HT - 1) / HT);
    if (blocks > sm_count() * 8) blocks = sm_count() * 8;
    cudaStream_t st = (cudaStream_t)stream;
    if (W == 1)
        hash_insert<1><<<blocks, HT, 0, st>>>(d_keys, n, d_table, (uint64_t)(slots - 1), d_n_new,
                                              d_status, spin_limit);
    else
        hash_insert<2><<<blocks, HT, 0, st>>>(d_keys, n, d_table, (uint64_t)(slots - 1), d_n_new,
                                              d_status, spin_limit);
    CUSCI_LAUNCHED(1, "hash insert probe");
    return CUSCI_OK;
}
