// System construction: device-resident integral tables and the per-eps
// screening bitmasks.
//
// The paper's excitation tables (Sec. 4.2.1, T_single and T_double) pad, per
// source orbital (pair), the list of target orbitals with their matrix element.
// A single excitation's element depends on every occupied orbital, so it cannot
// be stored per (p, a) exactly; here singles are summed on the fly from the
// slabs S1/S2, and doubles -- whose element depends only on (i, j, a, b) -- are
// read from the permuted slab T, with the screening decision precomputed as
// one bitmask word per (pair, a): bit b set iff |T| > eps.

#include <stdlib.h>
#include <string.h>

#include "cusci_internal.cuh"

namespace cusci {
namespace {

__global__ void build_small_tables(int n, const double *__restrict__ h2, double *J, double *K,
                                   double *S1, double *S2) {
    const size_t n2 = (size_t)n * n, n3 = n2 * n;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n3;
         t += (size_t)gridDim.x * blockDim.x) {
        int pk = (int)(t % n), pi = (int)((t / n) % n), pa = (int)(t / n2);
        // (pa pi | pk pk) and (pa pk | pk pi)
        S1[t] = h2[((size_t)(pa * n + pi) * n + pk) * n + pk];
        S2[t] = h2[((size_t)(pa * n + pk) * n + pk) * n + pi];
        if (t < n2) {
            int q = (int)(t % n), p = (int)(t / n);
            J[t] = h2[((size_t)(p * n + p) * n + q) * n + q];
            K[t] = h2[((size_t)(p * n + q) * n + q) * n + p];
        }
    }
}

// T: slab q = (kind*n + pi)*n + pj of `slab` doubles, element pa*n + pb
__global__ void build_T(int n, int slab, const double *__restrict__ h2, double *T) {
    const size_t total = 2 * (size_t)n * n * slab;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
         t += (size_t)gridDim.x * blockDim.x) {
        const size_t q = t / slab;
        const int e = (int)(t % slab);
        double v = 0.0;
        if (e < n * n) {
            const int pa = e / n, pb = e % n;
            const int pj = (int)(q % n), pi = (int)((q / n) % n), kind = (int)(q / ((size_t)n * n));
            const double direct = h2[((size_t)(pa * n + pi) * n + pb) * n + pj];  // (ai|bj)
            if (kind == 1) {
                v = direct;
            } else if (pi < pj && pa < pb) {
                const double exch = h2[((size_t)(pa * n + pj) * n + pb) * n + pi];  // (aj|bi)
                v = __dsub_rn(direct, exch);
            }
        }
        T[t] = v;
    }
}

__global__ void build_masks(int n, int slab, int mrow, const double *__restrict__ T, double eps,
                            uint64_t *bits) {
    const size_t rows = 2 * (size_t)n * n * mrow;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < rows;
         t += (size_t)gridDim.x * blockDim.x) {
        const size_t q = t / mrow;
        const int pa = (int)(t % mrow);
        const int pj = (int)(q % n), pi = (int)((q / n) % n), kind = (int)(q / ((size_t)n * n));
        uint64_t m = 0;
        if (pa < n && (kind == 1 || pi < pj)) {
            const double *row = T + q * slab + (size_t)pa * n;
            for (int pb = (kind == 0 ? pa + 1 : 0); pb < n; pb++)
                if (fabs(row[pb]) > eps) m |= 1ull << pb;
        }
        bits[t] = m;
    }
}

}  // namespace

size_t mask_words(const cusci_system *sys) {
    return 2 * (size_t)sys->norb * sys->norb * sys->mrow;
}

cusci_status build_masks_into(const cusci_system *sys, double eps, cudaStream_t stream,
                              uint64_t *bits) {
    const size_t rows = mask_words(sys);
    int blocks = (int)((rows + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    build_masks<<<blocks, 256, 0, stream>>>(sys->norb, sys->slab, sys->mrow, sys->T, eps, bits);
    CUSCI_LAUNCHED(1, "build_masks");
    return CUSCI_OK;
}

cusci_status masks_for(cusci_system *sys, double eps, cudaStream_t stream, const uint64_t **out) {
    uint64_t eps_bits;
    memcpy(&eps_bits, &eps, 8);
    for (int k = 0; k < CUSCI_MASK_SLOTS; k++) {
        MaskSlot &m = sys->masks[k];
        uint64_t mb;
        memcpy(&mb, &m.eps, 8);
        if (m.valid && mb == eps_bits) {
            m.stamp = ++sys->clock;
            *out = m.bits;
            return CUSCI_OK;
        }
    }
    // an unused slot, else the least recently used one
    int victim = -1;
    for (int k = 0; k < CUSCI_MASK_SLOTS && victim < 0; k++)
        if (!sys->masks[k].valid) victim = k;
    if (victim < 0) {
        victim = 0;
        for (int k = 1; k < CUSCI_MASK_SLOTS; k++)
            if (sys->masks[k].stamp < sys->masks[victim].stamp) victim = k;
    }
    MaskSlot &m = sys->masks[victim];
    if (m.valid) {
        // The slot is rebuilt in place: kernels of earlier calls, on any stream,
        // may still read it, so they must finish first.  Not possible while a
        // stream is being captured (warm the four slots up before capturing).
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        cudaError_t e = cudaStreamIsCapturing(stream, &cs);
        if (e != cudaSuccess) return cuda_fail(e, "screening masks: capture query");
        if (cs != cudaStreamCaptureStatusNone)
            return fail(CUSCI_ERR_INVALID,
                        "screening masks: a fifth eps on one system during graph capture");
        e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return cuda_fail(e, "screening masks: drain before rebuild");
        m.valid = false;
    }
    if (!m.bits) {
        cudaError_t e = cudaMalloc(&m.bits, mask_words(sys) * sizeof(uint64_t));
        if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(screening masks)");
    }
    cusci_status rc = build_masks_into(sys, eps, stream, m.bits);
    if (rc != CUSCI_OK) return rc;
    m.eps = eps;
    m.valid = true;
    m.stamp = ++sys->clock;
    *out = m.bits;
    return CUSCI_OK;
}

}  // namespace cusci

using namespace cusci;

extern "C" cusci_status cusci_system_create(int norb, int n_alpha, int n_beta, const double *h1,
                                            const double *h2, double ecore, cusci_system **out) {
    if (!out) return fail(CUSCI_ERR_INVALID, "cusci_system_create: out is NULL");
    *out = NULL;
    if (norb < 1 || norb > CUSCI_MAX_NORB)
        return fail(CUSCI_ERR_UNSUPPORTED, "cusci_system_create: norb=%d outside [1, %d]", norb,
                    CUSCI_MAX_NORB);
    if (n_alpha < 0 || n_beta < 0 || n_alpha > norb || n_beta > norb)
        return fail(CUSCI_ERR_INVALID, "cusci_system_create: n_alpha=%d n_beta=%d norb=%d",
                    n_alpha, n_beta, norb);
    if (!h1 || !h2) return fail(CUSCI_ERR_INVALID, "cusci_system_create: NULL integrals");

    cusci_system *s = (cusci_system *)calloc(1, sizeof(cusci_system));
    if (!s) return fail(CUSCI_ERR_OOM, "cusci_system_create: host allocation");
    s->norb = norb; s->n_alpha = n_alpha; s->n_beta = n_beta;
    s->M = 2 * norb; s->W = (2 * norb + 63) / 64; s->ecore = ecore;
    s->slab = norb * norb + ((norb * norb) & 1);
    s->mrow = norb + (norb & 1);
    cudaGetDevice(&s->device);

    const size_t n = norb, n2 = n * n, n3 = n2 * n, n4 = n3 * n;
    double *d_h2 = NULL;
    cudaError_t e;
#define ALLOC(ptr, cnt)                                                  \
    e = cudaMalloc(&(ptr), (cnt) * sizeof(double));                     \
    if (e != cudaSuccess) {                                              \
        cudaFree(d_h2);                                                  \
        cusci_system_destroy(s);                                         \
        return cuda_fail(e, "cusci_system_create: cudaMalloc");         \
    }
    ALLOC(s->h1, n2);
    ALLOC(s->J, n2);
    ALLOC(s->K, n2);
    ALLOC(s->S1, n3);
    ALLOC(s->S2, n3);
    ALLOC(s->T, 2 * n2 * (size_t)s->slab);
    ALLOC(d_h2, n4);
#undef ALLOC
    e = cudaMemcpy(s->h1, h1, n2 * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_h2, h2, n4 * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        int blocks = (int)((2 * n2 * (size_t)s->slab + 255) / 256);
        if (blocks > 8192) blocks = 8192;
        build_small_tables<<<(int)((n3 + 255) / 256), 256>>>(norb, d_h2, s->J, s->K, s->S1, s->S2);
        build_T<<<blocks, 256>>>(norb, s->slab, d_h2, s->T);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(0);
    cudaFree(d_h2);
    if (e != cudaSuccess) {
        cusci_system_destroy(s);
        return cuda_fail(e, "cusci_system_create: table build");
    }
    *out = s;
    return CUSCI_OK;
}

extern "C" void cusci_system_destroy(cusci_system *s) {
    if (!s) return;
    cudaFree(s->h1);
    cudaFree(s->J);
    cudaFree(s->K);
    cudaFree(s->S1);
    cudaFree(s->S2);
    cudaFree(s->T);
    for (int k = 0; k < CUSCI_MASK_SLOTS; k++) cudaFree(s->masks[k].bits);
    free(s);
}

extern "C" int cusci_system_words(const cusci_system *s) { return s ? s->W : 0; }
