// Local-energy form of the SCI energy (Eq. 5) over the coupled lists and the
// reverse index (Stage 3, Sec. 3):
//   y_i = sum_{e in row i} H_e psi_u[inverse[e]],   psi_i = psi_u[inverse[row start]]
//   E   = sum_i psi_i y_i / sum_i psi_i^2
// with psi given on the distinct coupled set U.  Forward: one warp per row,
// entries read coalesced, psi gathered through the inverse (four loads in
// flight per lane), a fixed shuffle tree per row and a fixed-order block
// reduction of the row terms (deterministic).  Adjoint:
//   dE/dpsi_u[u] = ( sum_{e: inverse[e]=u} psi_{i(e)} H_e
//                    + sum_{i: source of i is u} (y_i - 2 E psi_i) ) / sum psi_i^2
// a scatter-add into U in 128-bit fixed point (binary point at bit 64): every
// contribution psi_i H_e (and y_i - 2 E psi_i) is split into an integer and a
// 64-bit fraction and added with two integer atomics (the fraction's carry
// counted exactly once), so the sum is exact up to the 2^-64 truncation of each
// term and does not depend on the order of the additions -- the gradient is
// bit-reproducible run to run.  The common factor g / sum psi^2 is applied once
// per distinct configuration at the end.

#include "cusci_internal.cuh"

namespace cusci {
namespace {

constexpr int LW = 8;     // warps per block
constexpr int LU = 4;     // entries in flight per lane
constexpr int RED = 1024;

template <typename IDX>
__global__ void __launch_bounds__(32 * LW)
    le_rows(const int64_t *__restrict__ off, int64_t n, const double *__restrict__ h,
            const IDX *__restrict__ inv, const double *__restrict__ psi_u,
            double *__restrict__ y, double *__restrict__ pq) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (int64_t)blockIdx.x * LW + (threadIdx.x >> 5);
    const int64_t nw = (int64_t)gridDim.x * LW;
    for (int64_t i = warp; i < n; i += nw) {
        const int64_t b = off[i], e = off[i + 1];
        double acc = 0.0;
        for (int64_t k0 = b + lane; k0 < e; k0 += 32 * LU) {
            double hv[LU], pv[LU];
#pragma unroll
            for (int u = 0; u < LU; u++) {
                const int64_t k = k0 + 32 * u;
                hv[u] = 0.0;
                pv[u] = 0.0;
                if (k < e) {
                    hv[u] = h[k];
                    pv[u] = __ldg(psi_u + (int64_t)inv[k]);
                }
            }
#pragma unroll
            for (int u = 0; u < LU; u++) acc = __dadd_rn(acc, __dmul_rn(hv[u], pv[u]));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc = __dadd_rn(acc, __shfl_xor_sync(0xffffffffu, acc, o));
        if (lane == 0) {
            const double p = b < e ? __ldg(psi_u + (int64_t)inv[b]) : 0.0;
            if (y) y[i] = acc;
            pq[2 * i] = __dmul_rn(p, acc);
            pq[2 * i + 1] = __dmul_rn(p, p);
        }
    }
}

__device__ __forceinline__ void neumaier(double &sum, double &comp, double x) {
    const double t = __dadd_rn(sum, x);
    if (fabs(sum) >= fabs(x)) comp = __dadd_rn(comp, __dadd_rn(__dsub_rn(sum, t), x));
    else comp = __dadd_rn(comp, __dadd_rn(__dsub_rn(x, t), sum));
    sum = t;
}

// one block, fixed order: E = sum pq[2i] / sum pq[2i+1]
__global__ void __launch_bounds__(RED)
    le_reduce(const double *__restrict__ pq, int64_t n, double *__restrict__ E,
              double *__restrict__ norm2) {
    __shared__ double sn[RED], sd[RED];
    double ns = 0.0, nc = 0.0, ds = 0.0, dc = 0.0;
    const int64_t per = (n + RED - 1) / RED;
    const int64_t b = threadIdx.x * per;
    const int64_t e = b + per < n ? b + per : n;
    for (int64_t i = b; i < e; i++) {
        neumaier(ns, nc, pq[2 * i]);
        neumaier(ds, dc, pq[2 * i + 1]);
    }
    sn[threadIdx.x] = __dadd_rn(ns, nc);
    sd[threadIdx.x] = __dadd_rn(ds, dc);
    __syncthreads();
    for (int o = RED / 2; o > 0; o >>= 1) {
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

// adds c (|c| < 2^62) to the 128-bit fixed-point accumulator a[0] (fraction,
// 2^-64 units) / a[1] (two's-complement integer part)
__device__ __forceinline__ void fx_add(unsigned long long *a, double c) {
    const double f = floor(c);
    const long long ip = __double2ll_rz(f);                 // exact
    const double frac = __dsub_rn(c, f);                      // exact, in [0, 1)
    const unsigned long long lo = __double2ull_rz(__dmul_rn(frac, 18446744073709551616.0));
    const unsigned long long old = atomicAdd(a, lo);
    const unsigned long long carry = old + lo < old ? 1ull : 0ull;
    // the high word changes only by ip + carry: zero for a term in [0, 1)
    // without a carry, and for a term in [-1, 0) whose low word wrapped
    const unsigned long long hi = (unsigned long long)ip + carry;
    if (hi != 0ull) atomicAdd(a + 1, hi);
}

template <typename IDX>
__global__ void __launch_bounds__(32 * LW)
    le_scatter_fx(const int64_t *__restrict__ off, int64_t n, const double *__restrict__ h,
                  const IDX *__restrict__ inv, const double *__restrict__ psi_u,
                  const double *__restrict__ y, const double *__restrict__ E,
                  unsigned long long *__restrict__ acc) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (int64_t)blockIdx.x * LW + (threadIdx.x >> 5);
    const int64_t nw = (int64_t)gridDim.x * LW;
    const double e2 = __dmul_rn(2.0, *E);
    for (int64_t i = warp; i < n; i += nw) {
        const int64_t b = off[i], e = off[i + 1];
        if (b >= e) continue;
        const int64_t s = (int64_t)inv[b];
        const double p = __ldg(psi_u + s);
        for (int64_t k = b + lane; k < e; k += 32)
            fx_add(acc + 2 * (int64_t)inv[k], __dmul_rn(p, h[k]));
        if (lane == 0) fx_add(acc + 2 * s, __dsub_rn(y[i], __dmul_rn(e2, p)));
    }
}

// grad_u[u] = (g / sum psi^2) * (integer part + fraction) of the accumulator
__global__ void le_finish_fx(const unsigned long long *__restrict__ acc, int64_t nu,
                             const double *__restrict__ norm2, const double *__restrict__ gout,
                             double *__restrict__ grad_u) {
    const double scale = __ddiv_rn(gout ? *gout : 1.0, *norm2);
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < nu;
         u += (int64_t)gridDim.x * blockDim.x) {
        const double v = __dadd_rn(__ll2double_rn((long long)acc[2 * u + 1]),
                                   __dmul_rn(__ull2double_rn(acc[2 * u]), 5.421010862427522e-20));
        grad_u[u] = __dmul_rn(scale, v);
    }
}

size_t al(size_t x) { return (x + 255) & ~(size_t)255; }

cusci_status check_args(const int64_t *off, int64_t n, const double *h, const void *inv,
                        int index_bytes, const double *psi_u, const char *who) {
    if (n < 1 || !off || !h || !inv || !psi_u)
        return fail(CUSCI_ERR_INVALID, "%s: bad argument (n must be >= 1)", who);
    if (index_bytes != 4 && index_bytes != 8)
        return fail(CUSCI_ERR_INVALID, "%s: index_bytes must be 4 or 8", who);
    return CUSCI_OK;
}

}  // namespace
}  // namespace cusci

using namespace cusci;

extern "C" cusci_status cusci_local_energy_workspace(int64_t n, size_t *bytes) {
    if (!bytes || n < 0) return fail(CUSCI_ERR_INVALID, "cusci_local_energy_workspace: bad argument");
    *bytes = al((size_t)(n > 0 ? n : 1) * 16) + al((size_t)(n > 0 ? n : 1) * 8);
    return CUSCI_OK;
}

extern "C" cusci_status cusci_local_energy_fwd(const int64_t *d_offsets, int64_t n,
                                               const double *d_h, const void *d_inverse,
                                               int index_bytes, const double *d_psi_u,
                                               double *d_y, double *d_E, double *d_norm2,
                                               void *d_ws, size_t ws_bytes, void *stream) {
    cusci_status rc = check_args(d_offsets, n, d_h, d_inverse, index_bytes, d_psi_u,
                                 "cusci_local_energy_fwd");
    if (rc != CUSCI_OK) return rc;
    if (!d_E || !d_norm2) return fail(CUSCI_ERR_INVALID, "cusci_local_energy_fwd: NULL output");
    size_t need = 0;
    cusci_local_energy_workspace(n, &need);
    if (!d_ws || ws_bytes < need)
        return fail(CUSCI_ERR_OOM, "cusci_local_energy_fwd: workspace %zu < %zu", ws_bytes, need);
    if ((uintptr_t)d_ws & 255u) return fail(CUSCI_ERR_INVALID, "local energy: workspace alignment");
    cudaStream_t st = (cudaStream_t)stream;
    double *pq = (double *)d_ws;
    double *yw = d_y ? d_y : (double *)((unsigned char *)d_ws + al((size_t)n * 16));
    const int grid = sm_count() * 8;
    if (index_bytes == 4)
        le_rows<int32_t><<<grid, 32 * LW, 0, st>>>(d_offsets, n, d_h, (const int32_t *)d_inverse,
                                                   d_psi_u, yw, pq);
    else
        le_rows<int64_t><<<grid, 32 * LW, 0, st>>>(d_offsets, n, d_h, (const int64_t *)d_inverse,
                                                   d_psi_u, yw, pq);
    le_reduce<<<1, RED, 0, st>>>(pq, n, d_E, d_norm2);
    CUSCI_LAUNCHED(2, "local energy forward");
    return CUSCI_OK;
}

extern "C" cusci_status cusci_local_energy_bwd_workspace(int64_t n, int64_t n_unique,
                                                         size_t *bytes) {
    if (!bytes || n < 0 || n_unique < 0)
        return fail(CUSCI_ERR_INVALID, "cusci_local_energy_bwd_workspace: bad argument");
    size_t rows = 0;
    cusci_local_energy_workspace(n, &rows);
    *bytes = rows + al((size_t)(n_unique > 0 ? n_unique : 1) * 16);
    return CUSCI_OK;
}

extern "C" cusci_status cusci_local_energy_bwd(const int64_t *d_offsets, int64_t n,
                                               const double *d_h, const void *d_inverse,
                                               int index_bytes, const double *d_psi_u,
                                               int64_t n_unique, const double *d_y,
                                               const double *d_E, const double *d_norm2,
                                               const double *d_grad_out, double *d_grad_u,
                                               void *d_ws, size_t ws_bytes, void *stream) {
    cusci_status rc = check_args(d_offsets, n, d_h, d_inverse, index_bytes, d_psi_u,
                                 "cusci_local_energy_bwd");
    if (rc != CUSCI_OK) return rc;
    if (!d_E || !d_norm2 || !d_grad_u || n_unique < 1)
        return fail(CUSCI_ERR_INVALID, "cusci_local_energy_bwd: bad output");
    cudaStream_t st = (cudaStream_t)stream;
    const int grid = sm_count() * 8;
    size_t need = 0, rows = 0;
    cusci_local_energy_bwd_workspace(n, n_unique, &need);
    cusci_local_energy_workspace(n, &rows);
    if (!d_ws || ws_bytes < need)
        return fail(CUSCI_ERR_OOM, "cusci_local_energy_bwd: workspace %zu < %zu", ws_bytes, need);
    if ((uintptr_t)d_ws & 255u) return fail(CUSCI_ERR_INVALID, "local energy: workspace alignment");
    const double *y = d_y;
    if (!y) {
        double *pq = (double *)d_ws;
        double *yw = (double *)((unsigned char *)d_ws + al((size_t)n * 16));
        if (index_bytes == 4)
            le_rows<int32_t><<<grid, 32 * LW, 0, st>>>(d_offsets, n, d_h,
                                                       (const int32_t *)d_inverse, d_psi_u, yw, pq);
        else
            le_rows<int64_t><<<grid, 32 * LW, 0, st>>>(d_offsets, n, d_h,
                                                       (const int64_t *)d_inverse, d_psi_u, yw, pq);
        CUSCI_LAUNCHED(1, "local energy: rows");
        y = yw;
    }
    unsigned long long *acc = (unsigned long long *)((unsigned char *)d_ws + rows);
    cudaError_t e = cudaMemsetAsync(acc, 0, (size_t)n_unique * 16, st);
    if (e != cudaSuccess) return cuda_fail(e, "local energy: clear accumulators");
    if (index_bytes == 4)
        le_scatter_fx<int32_t><<<grid, 32 * LW, 0, st>>>(d_offsets, n, d_h,
                                                         (const int32_t *)d_inverse, d_psi_u, y,
                                                         d_E, acc);
    else
        le_scatter_fx<int64_t><<<grid, 32 * LW, 0, st>>>(d_offsets, n, d_h,
                                                         (const int64_t *)d_inverse, d_psi_u, y,
                                                         d_E, acc);
    le_finish_fx<<<sm_count() * 4, 256, 0, st>>>(acc, n_unique, d_norm2, d_grad_out, d_grad_u);
    CUSCI_LAUNCHED(2, "local energy backward");
    CUSCI_LAUNCHED(2, "local energy backward");
    return CUSCI_OK;
}
