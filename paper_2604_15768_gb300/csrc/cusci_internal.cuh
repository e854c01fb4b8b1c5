// Internal declarations shared by the libcusci translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/cusci.h"

#define CUSCI_MAX_NORB 64
#define CUSCI_MASK_SLOTS 4

namespace cusci {

// One cached set of screening bitmasks for a given eps.
// bits[((kind*norb + pi)*norb + pj)*mrow + pa] has bit pb set iff the double
// excitation with spatial occupied (pi, pj) and virtual (pa, pb) survives
// |H| > eps; kind 0 = both electrons of one spin (only pi < pj, pa < pb are
// set), kind 1 = opposite spins.
struct MaskSlot {
    double eps;
    uint64_t *bits;
    uint64_t stamp;
    bool valid;
};

}  // namespace cusci

struct cusci_system {
    int norb, n_alpha, n_beta, W, M;
    double ecore;
    int device;
    // device tables, all FP64, spatial indices
    double *h1;   // [p][q]
    double *J;    // [p][q] = (pp|qq)
    double *K;    // [p][q] = (pq|qp)
    double *S1;   // [pa][pi][pk] = (pa pi|pk pk)
    double *S2;   // [pa][pi][pk] = (pa pk|pk pi)
    double *T;    // [kind][pi][pj] slabs of `slab` doubles, element [pa*norb + pb]:
                  // kind 0 (ai|bj)-(aj|bi), kind 1 (ai|bj)
    int slab;     // norb^2 rounded up to even (16-byte slabs for bulk copies)
    int mrow;     // norb rounded up to even (16-byte mask rows)
    cusci::MaskSlot masks[CUSCI_MASK_SLOTS];
    uint64_t clock;
};

namespace cusci {

// number of kernel launches issued by the library (capi.cu)
void note_launches(int n);

// thread-local error message plumbing (capi.cu)
cusci_status fail(cusci_status st, const char *fmt, ...);
cusci_status cuda_fail(cudaError_t e, const char *what);

// raises fn's dynamic shared-memory limit to >= bytes on the current device
// (once per function and device, thread-safe)
cusci_status allow_smem(const void *fn, size_t bytes, const char *what);

// returns the screening masks for eps, building them on `stream` if needed
// (the system keeps CUSCI_MASK_SLOTS of them, least recently used replaced;
// replacing one first waits for the device's earlier work)
cusci_status masks_for(cusci_system *sys, double eps, cudaStream_t stream,
                       const uint64_t **out);
// words of one set of screening masks, and a build of one into caller memory
size_t mask_words(const cusci_system *sys);
cusci_status build_masks_into(const cusci_system *sys, double eps, cudaStream_t stream,
                              uint64_t *bits);

// device view of a system for kernels
struct SysView {
    int norb, M, W, slab, mrow;
    double ecore;
    const double *__restrict__ h1;
    const double *__restrict__ J;
    const double *__restrict__ K;
    const double *__restrict__ S1;
    const double *__restrict__ S2;
    const double *__restrict__ T;
    const uint64_t *__restrict__ mask;
};

inline SysView view_of(const cusci_system *s, const uint64_t *mask) {
    SysView v;
    v.norb = s->norb; v.M = s->M; v.W = s->W; v.ecore = s->ecore;
    v.slab = s->slab; v.mrow = s->mrow;
    v.h1 = s->h1; v.J = s->J; v.K = s->K; v.S1 = s->S1; v.S2 = s->S2; v.T = s->T;
    v.mask = mask;
    return v;
}

inline int sm_count() {
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

}  // namespace cusci

#define CUSCI_CHECK_LAUNCH(what)                                   \
    do {                                                          \
        cudaError_t _e = cudaGetLastError();                      \
        if (_e != cudaSuccess) return cusci::cuda_fail(_e, what); \
    } while (0)

// launches `n` kernels' worth of bookkeeping, then checks the launch status
#define CUSCI_LAUNCHED(n, what)   \
    do {                          \
        cusci::note_launches(n);  \
        CUSCI_CHECK_LAUNCH(what); \
    } while (0)
