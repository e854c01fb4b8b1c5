// Variational energy over a selected set S and its adjoint.
//
// E = psi.(H psi) / psi.psi (Eq. 1 restricted to S, Sec. 2.1), with
// (H psi)_i = sum_{j in C_i, j in S} H_ij psi_j.  The coupled lists are
// regenerated per row by the same warp enumeration as the fill pass and never
// stored; membership j in S is resolved just in time (Stage 3, Sec. 4.3) in an
// open-addressing hash table of S built in the caller's workspace (S is 1.6 MB
// of keys for 200k determinants, so the table stays in L2).  An exact
// prefilter skips the probe for targets farther from S[0] -- per spin or in
// total -- than every member of S, and a one-bit-per-hash filter of S (16 bits
// per member, L2-resident) skips it for almost every other non-member.
// Reductions are deterministic: per-row warp shuffles in a fixed pattern, then
// one block that sums rows in a fixed order (Neumaier-compensated per thread)
// followed by a fixed tree -- no floating-point atomics.
// Adjoint: dE/dpsi_i = 2 ((H psi)_i - E psi_i) / psi.psi, scaled by the
// incoming gradient; H psi is taken from the forward pass or recomputed.

#include "enumerate.cuh"

namespace cusci {
namespace {

using namespace enumr;
constexpr int EW = 8;  // warps per block

// multiplicative (Fibonacci) hash: top bits of the product select the slot
template <int W>
__device__ __forceinline__ uint64_t hash_det(const uint64_t *d, int shift) {
    uint64_t x = d[0];
    if (W == 2) x ^= d[W - 1] * 0xc2b2ae3d27d4eb4full;
    return (x * 0x9e3779b97f4a7c15ull) >> shift;
}

struct Table {
    uint64_t *keys;   // [cap][W]
    int64_t *vals;    // [cap], 0 = empty, else index + 1
    uint64_t mask;    // cap - 1
    int shift;        // 64 - log2(cap)
    const uint64_t *ref;       // S[0]
    const uint32_t *maxdist;   // [3]: largest alpha, beta and total distance of S from S[0]
    uint32_t *bloom;           // one bit per 2^-bshift of a second hash: set for every member
    int bshift;                // 64 - log2(bloom bits)
};

// the filter bit of a determinant: a second multiplicative hash, independent
// of the table slot; a clear bit proves the determinant is not in S
template <int W>
__device__ __forceinline__ uint64_t bloom_bit(const uint64_t *d, int bshift) {
    uint64_t x = d[0];
    if (W == 2) x ^= d[W - 1] * 0x9fb21c651e98df25ull;
    return (x * 0xd6e8feb86659fd93ull) >> bshift;
}

// occupation differences of t from the reference, per spin
template <int W>
__device__ __forceinline__ void spin_dist(const uint64_t *t, const uint64_t *ref, uint32_t &da,
                                          uint32_t &db) {
    da = 0;
    db = 0;
#pragma unroll
    for (int w = 0; w < W; w++) {
        const uint64_t x = t[w] ^ ref[w];
        da += __popcll(x & 0x5555555555555555ull);
        db += __popcll(x & 0xAAAAAAAAAAAAAAAAull);
    }
}

template <int W>
__global__ void insert_S(Table tb, const uint64_t *__restrict__ S, int64_t nS,
                         uint32_t *__restrict__ maxdist, int32_t *__restrict__ status) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nS;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t d[W];
#pragma unroll
        for (int q = 0; q < W; q++) d[q] = S[i * W + q];
        if (i > 0 && status) {
            // S must be strictly ascending (word W-1 most significant)
            bool gt = false, eq = true;
#pragma unroll
            for (int q = W - 1; q >= 0; q--) {
                uint64_t p = S[(i - 1) * W + q];
                if (eq && d[q] != p) {
                    gt = d[q] > p;
                    eq = false;
                }
            }
            if (!gt) *status = CUSCI_ERR_INVALID;
        }
        uint32_t da, db;
        spin_dist<W>(d, S, da, db);
        atomicMax(maxdist, da);
        atomicMax(maxdist + 1, db);
        atomicMax(maxdist + 2, da + db);
        const uint64_t bb = bloom_bit<W>(d, tb.bshift);
        atomicOr(tb.bloom + (bb >> 5), 1u << (bb & 31));
        uint64_t h = hash_det<W>(d, tb.shift);
        for (uint64_t probe = 0; probe <= tb.mask; probe++) {
            unsigned long long old =
                atomicCAS((unsigned long long *)(tb.vals + h), 0ull, (unsigned long long)(i + 1));
            if (old == 0ull) {
#pragma unroll
                for (int q = 0; q < W; q++) tb.keys[h * W + q] = d[q];
                break;
            }
            h = (h + 1) & tb.mask;
        }
    }
}

template <int W>
__device__ __forceinline__ int64_t lookup(const Table &tb, const uint64_t (&t)[W]) {
    // exact prefilter: a target farther from S[0] (per spin) than every member
    // of S cannot be in S
    uint32_t da, db;
    spin_dist<W>(t, tb.ref, da, db);
    if (da > __ldg(tb.maxdist) || db > __ldg(tb.maxdist + 1) || da + db > __ldg(tb.maxdist + 2))
        return -1;
    // most targets are not in S: one filter word (L1/L2) instead of a probe sequence
    const uint64_t bb = bloom_bit<W>(t, tb.bshift);
    if (!((__ldg(tb.bloom + (bb >> 5)) >> (bb & 31)) & 1u)) return -1;
    uint64_t h = hash_det<W>(t, tb.shift);
    for (uint64_t probe = 0; probe <= tb.mask; probe++) {
        const int64_t v = __ldg(tb.vals + h);
        if (v == 0) return -1;
        bool eq = true;
#pragma unroll
        for (int q = 0; q < W; q++) eq &= __ldg(tb.keys + h * W + q) == t[q];
        if (eq) return v - 1;
        h = (h + 1) & tb.mask;
    }
    return -1;
}

template <int W>
struct HpsiEmit {
    const Table *tb;
    const double *__restrict__ psi;
    double acc;
    // every target of the pair / row toggles `flips` more bits (a, b), each of
    // which can shorten its distance to S[0] by at most one: if even then it is
    // farther than every member of S, none of them is in S
    __device__ __forceinline__ bool within(const uint64_t (&t)[W], int fa, int fb) const {
        uint32_t da, db;
        spin_dist<W>(t, tb->ref, da, db);
        const uint32_t ma = __ldg(tb->maxdist), mb = __ldg(tb->maxdist + 1),
                       mt = __ldg(tb->maxdist + 2);
        return (int)da - fa <= (int)ma && (int)db - fb <= (int)mb &&
               (int)(da + db) - fa - fb <= (int)mt;
    }
    __device__ __forceinline__ bool pair_possible(const uint64_t (&t)[W], int si, int sj) const {
        return within(t, (si == 0) + (sj == 0), (si == 1) + (sj == 1));
    }
    __device__ __forceinline__ bool row_possible(const uint64_t (&t)[W], int sj) const {
        return within(t, sj == 0, sj == 1);
    }
    __device__ __forceinline__ void operator()(const uint64_t (&t)[W], double h, int64_t) {
        const int64_t j = lookup<W>(*tb, t);
        if (j >= 0) acc = __dadd_rn(acc, __dmul_rn(h, __ldg(psi + j)));
    }
};

template <int W>
__global__ void __launch_bounds__(32 * EW)
    hpsi_kernel(SysView v, Table tb, const uint64_t *__restrict__ S, int64_t nS, double eps,
                const double *__restrict__ psi, double *__restrict__ hpsi) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (int64_t)blockIdx.x * EW + (threadIdx.x >> 5);
    const int64_t nwarps = (int64_t)gridDim.x * EW;
    for (int64_t i = warp; i < nS; i += nwarps) {
        Src<W> s;
        decode<W>(S + i * W, v.norb, s);
        HpsiEmit<W> em{&tb, psi, 0.0};
        visit_source<W>(v, s, eps, lane, em);
        double a = em.acc;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a = __dadd_rn(a, __shfl_xor_sync(FULL, a, o));
        if (lane == 0) hpsi[i] = a;
    }
}

constexpr int RED_T = 1024;

__device__ __forceinline__ void neumaier_add(double &sum, double &comp, double x) {
    const double t = __dadd_rn(sum, x);
    if (fabs(sum) >= fabs(x)) comp = __dadd_rn(comp, __dadd_rn(__dsub_rn(sum, t), x));
    else comp = __dadd_rn(comp, __dadd_rn(__dsub_rn(x, t), sum));
    sum = t;
}

// one block: E = sum psi*hpsi / sum psi^2, fixed order
__global__ void __launch_bounds__(RED_T)
    reduce_energy(const double *__restrict__ psi, const double *__restrict__ hpsi, int64_t nS,
                  double *__restrict__ E, double *__restrict__ norm2) {
    __shared__ double sn[RED_T], sd[RED_T];
    double ns = 0.0, nc = 0.0, ds = 0.0, dc = 0.0;
    // contiguous chunk per thread keeps the order fixed for a given nS
    const int64_t per = (nS + RED_T - 1) / RED_T;
    const int64_t b = threadIdx.x * per;
    int64_t e = b + per;
    if (e > nS) e = nS;
    for (int64_t i = b; i < e; i++) {
        const double p = psi[i];
        neumaier_add(ns, nc, __dmul_rn(p, hpsi[i]));
        neumaier_add(ds, dc, __dmul_rn(p, p));
    }
    sn[threadIdx.x] = __dadd_rn(ns, nc);
    sd[threadIdx.x] = __dadd_rn(ds, dc);
    __syncthreads();
    for (int o = RED_T / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            sn[threadIdx.x] = __dadd_rn(sn[threadIdx.x], sn[threadIdx.x + o]);
            sd[threadIdx.x] = __dadd_rn(sd[threadIdx.x], sd[threadIdx.x + o]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        *norm2 = sd[0];
        *E = __ddiv_rn(sn[0], sd[0]);
    }
}

__global__ void grad_kernel(const double *__restrict__ psi, const double *__restrict__ hpsi,
                            int64_t nS, const double *__restrict__ E,
                            const double *__restrict__ norm2, const double *__restrict__ gout,
                            double *__restrict__ grad) {
    const double e = *E, n2 = *norm2, g = gout ? *gout : 1.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nS;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double r = __dsub_rn(hpsi[i], __dmul_rn(e, psi[i]));
        grad[i] = __dmul_rn(g, __ddiv_rn(__dmul_rn(2.0, r), n2));
    }
}

uint64_t table_cap(int64_t nS) {
    uint64_t cap = 1024;
    while (cap < (uint64_t)(2 * nS)) cap <<= 1;
    return cap;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct EPlan {
    uint64_t cap;
    int log2cap, log2bloom;
    size_t off_keys, off_vals, off_hp, off_md, off_bloom, bytes;
};

EPlan eplan(int64_t nS, int W) {
    EPlan p;
    p.cap = table_cap(nS);
    p.log2cap = 0;
    while ((1ull << p.log2cap) < p.cap) p.log2cap++;
    size_t off = 0;
    p.off_keys = off; off = align256(off + p.cap * 8 * W);
    p.off_vals = off; off = align256(off + p.cap * 8);
    p.off_hp = off; off = align256(off + (size_t)(nS > 0 ? nS : 1) * 8);
    p.off_md = off; off = align256(off + 16);
    // filter: a power of two of at least 16 bits per member (false positives
    // about 6%), at least 2^12 bits
    p.log2bloom = 12;
    while ((1ull << p.log2bloom) < (uint64_t)(nS > 0 ? nS : 1) * 16) p.log2bloom++;
    p.off_bloom = off; off = align256(off + ((size_t)1 << p.log2bloom) / 8);
    p.bytes = off;
    return p;
}

cusci_status compute_hpsi(const cusci_system *sys, const uint64_t *d_S, int64_t nS,
                          const double *d_psi, double eps, double *hp, void *d_ws,
                          size_t ws_bytes, int32_t *d_status, cudaStream_t st) {
    const EPlan p = eplan(nS, sys->W);
    if (!d_ws || ws_bytes < p.bytes)
        return fail(CUSCI_ERR_OOM, "energy: workspace %zu < %zu bytes", ws_bytes, p.bytes);
    if ((uintptr_t)d_ws & 255u) return fail(CUSCI_ERR_INVALID, "energy: workspace not 256-aligned");
    unsigned char *ws = (unsigned char *)d_ws;
    uint32_t *md = (uint32_t *)(ws + p.off_md);
    Table tb{(uint64_t *)(ws + p.off_keys), (int64_t *)(ws + p.off_vals), p.cap - 1,
             64 - p.log2cap, d_S, md, (uint32_t *)(ws + p.off_bloom), 64 - p.log2bloom};
    cudaError_t e = cudaMemsetAsync(tb.vals, 0, p.cap * 8, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(tb.bloom, 0, ((size_t)1 << p.log2bloom) / 8, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(md, 0, 16, st);
    if (e != cudaSuccess) return cuda_fail(e, "energy: table clear");
    const uint64_t *mask = NULL;
    cusci_status rc = masks_for(const_cast<cusci_system *>(sys), eps, st, &mask);
    if (rc != CUSCI_OK) return rc;
    SysView v = view_of(sys, mask);
    int ib = (int)((nS + 255) / 256);
    if (ib > sm_count() * 8) ib = sm_count() * 8;
    int64_t want = (nS + EW - 1) / EW;
    int grid = (int)(want < sm_count() * 8 ? want : sm_count() * 8);
    // unstaged: the hash probes are latency-bound, so full occupancy (64 warps
    // per SM) beats shared-memory staging of the integral slabs here
    if (sys->W == 1) {
        insert_S<1><<<ib, 256, 0, st>>>(tb, d_S, nS, md, d_status);
        hpsi_kernel<1><<<grid, 32 * EW, 0, st>>>(v, tb, d_S, nS, eps, d_psi, hp);
    } else {
        insert_S<2><<<ib, 256, 0, st>>>(tb, d_S, nS, md, d_status);
        hpsi_kernel<2><<<grid, 32 * EW, 0, st>>>(v, tb, d_S, nS, eps, d_psi, hp);
    }
    CUSCI_LAUNCHED(2, "energy: H psi");
    return CUSCI_OK;
}

}  // namespace
}  // namespace cusci

using namespace cusci;

extern "C" cusci_status cusci_energy_workspace(const cusci_system *sys, int64_t nS,
                                               size_t *bytes) {
    if (!sys || !bytes || nS < 0) return fail(CUSCI_ERR_INVALID, "cusci_energy_workspace: bad argument");
    *bytes = eplan(nS, sys->W).bytes;
    return CUSCI_OK;
}

extern "C" cusci_status cusci_energy_fwd(const cusci_system *sys, const uint64_t *d_S, int64_t nS,
                                         const double *d_psi, double eps, double *d_E,
                                         double *d_norm2, double *d_Hpsi, void *d_ws,
                                         size_t ws_bytes, int32_t *d_status, void *stream) {
    if (!sys || nS < 1 || !d_S || !d_psi || !d_E || !d_norm2)
        return fail(CUSCI_ERR_INVALID, "cusci_energy_fwd: bad argument (nS must be >= 1)");
    if (eps != eps) return fail(CUSCI_ERR_INVALID, "cusci_energy_fwd: eps is NaN");
    cudaStream_t st = (cudaStream_t)stream;
    const EPlan p = eplan(nS, sys->W);
    double *hp = d_Hpsi ? d_Hpsi : (double *)((unsigned char *)d_ws + p.off_hp);
    cusci_status rc = compute_hpsi(sys, d_S, nS, d_psi, eps, hp, d_ws, ws_bytes, d_status, st);
    if (rc != CUSCI_OK) return rc;
    reduce_energy<<<1, RED_T, 0, st>>>(d_psi, hp, nS, d_E, d_norm2);
    CUSCI_LAUNCHED(1, "energy: reduction");
    return CUSCI_OK;
}

extern "C" cusci_status cusci_energy_bwd(const cusci_system *sys, const uint64_t *d_S, int64_t nS,
                                         const double *d_psi, double eps, const double *d_E,
                                         const double *d_norm2, const double *d_Hpsi,
                                         const double *d_grad_out, double *d_grad, void *d_ws,
                                         size_t ws_bytes, void *stream) {
    if (!sys || nS < 1 || !d_S || !d_psi || !d_E || !d_norm2 || !d_grad)
        return fail(CUSCI_ERR_INVALID, "cusci_energy_bwd: bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    const double *hp = d_Hpsi;
    if (!hp) {
        const EPlan p = eplan(nS, sys->W);
        double *w = (double *)((unsigned char *)d_ws + p.off_hp);
        cusci_status rc = compute_hpsi(sys, d_S, nS, d_psi, eps, w, d_ws, ws_bytes, NULL, st);
        if (rc != CUSCI_OK) return rc;
        hp = w;
    }
    int blocks = (int)((nS + 255) / 256);
    if (blocks > sm_count() * 8) blocks = sm_count() * 8;
    grad_kernel<<<blocks, 256, 0, st>>>(d_psi, hp, nS, d_E, d_norm2, d_grad_out, d_grad);
    CUSCI_LAUNCHED(1, "energy: gradient");
    return CUSCI_OK;
}
