// Fixed device scratch for the matvec variant that allocates nothing
// (tdbem_hessenberg_apply_noalloc). The paper has no counterpart: this is a
// service for callers that cannot allocate device memory at the point of the
// product, for example a solver loop that has committed all device memory to
// its own pool, or code running under a fixed memory budget where an
// allocation could fail in the middle of a time-stepping run.
//
// The transposed x lives in one array of device global memory, reserved when
// the CUDA module of this file is loaded: MV_STATIC_MAX doubles (16 MiB), so
// N * M must not exceed 2^21 (the 20480-triangle sphere with 129 time points
// needs 1.32e6). Nothing in it has to start at zero: the transpose overwrites
// every entry that the product then reads. The array is shared by every call
// on the device, whatever the assembler, so calls that overlap in time (on
// different streams or host threads) race on it and must be ordered.
#include <mutex>

#include "tdbem_internal.h"

namespace tdbem {

static __device__ __align__(256) double g_mv_scratch[MV_STATIC_MAX];

namespace {
constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
double *g_scratch_ptr[MAX_DEVICES] = {};
}  // namespace

// Device address of the scratch on the current device, looked up once per
// device (with that device current) by the first call.
cudaError_t static_mv_scratch(double **ptr) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_mv_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = (double *)p;
    }
    *ptr = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace tdbem
