// Fixed device scratch for the matvec variant that allocates nothing
// (tdbem_hessenberg_apply_noalloc). The paper has no counterpart: this is a
// service for callers that cannot allocate device memory at the point of the
// product, for example a solver loop that has committed all device memory to
// its own pool, or code running under a fixed memory budget where an
// allocation could fail in the middle of a time-stepping run.
//
// The transposed x lives in one array of device global memory of
// MV_STATIC_MAX doubles (16 MiB), so N * M must not exceed 2^21 (the
// 20480-triangle sphere with 129 time points needs 1.32e6). The CUDA runtime
// loads this file's module, and with it reserves the array, lazily: on a
// device, the first call of the entry point does it, so a caller that plans
// to commit all remaining device memory to its own pool makes one call first
// (and makes the first call before any stream capture). Nothing in the array
// has to start at zero: the transpose overwrites every entry that the
// product then reads. The array is shared by every call on the device,
// whatever the assembler, so calls that overlap in time (on different
// streams or host threads) race on it and must be ordered.
#include "tdbem_internal.h"

namespace tdbem {

static __device__ __align__(256) double g_mv_scratch[MV_STATIC_MAX];

// Device address of the scratch on the current device, looked up on every
// call (with that device current): cheap once the module is loaded, and
// still right after a device reset reloads the module at a new address.
cudaError_t static_mv_scratch(double **ptr) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_mv_scratch);
    if (e != cudaSuccess) return e;
    *ptr = (double *)p;
    return cudaSuccess;
}

}  // namespace tdbem
