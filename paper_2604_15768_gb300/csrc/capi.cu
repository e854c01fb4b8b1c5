// Error reporting and version of the C ABI.
#include <atomic>
#include <map>
#include <mutex>
#include <stdarg.h>
#include <stdio.h>
#include <utility>

#include "cusci_internal.cuh"

namespace {
thread_local char g_last_error[512] = "";
std::atomic<unsigned long long> g_launches{0};
}

namespace cusci {

void note_launches(int n) { g_launches.fetch_add((unsigned long long)n); }

cusci_status fail(cusci_status st, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
    va_end(ap);
    return st;
}

cusci_status cuda_fail(cudaError_t e, const char *what) {
    return fail(e == cudaErrorMemoryAllocation ? CUSCI_ERR_OOM : CUSCI_ERR_CUDA, "%s: %s (%s)",
                what, cudaGetErrorString(e), cudaGetErrorName(e));
}

// Raises a kernel's dynamic shared-memory limit to at least `bytes` on the
// current device.  The attribute is per (function, device); the largest value
// set so far is remembered under a lock, so concurrent callers and several
// devices are safe.
cusci_status allow_smem(const void *fn, size_t bytes, const char *what) {
    static std::mutex mu;
    static std::map<std::pair<const void *, int>, size_t> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, what);
    std::lock_guard<std::mutex> lk(mu);
    size_t &have = done[std::make_pair(fn, dev)];
    if (have >= bytes) return CUSCI_OK;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return cuda_fail(e, what);
    have = bytes;
    return CUSCI_OK;
}

}  // namespace cusci

extern "C" const char *cusci_last_error(void) { return g_last_error; }
extern "C" const char *cusci_version(void) { return "cusci 0.1 (sm_103a)"; }
extern "C" uint64_t cusci_kernel_launches(void) { return (uint64_t)g_launches.load(); }
