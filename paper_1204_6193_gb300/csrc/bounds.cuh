// bounds.cuh -- the bounds-check build of the library (compiled with
// -DRNG_BOUNDS_CHECK into its own shared object, see build.py).
//
// RNGX_IDX_OK(i, n, site) is true when 0 <= i < n.  In a checked build an
// index outside [0, n) records `site` -- a number naming the access, file
// code * 10000 + line -- in this module's status word (the first violation
// is kept), and the caller skips the access, so that a wrong index becomes
// an error status the host reads (rng_debug_bounds_status) instead of a
// memory fault.  In the normal build the predicate is the constant true and
// the checks cost nothing.
//
// Each translation unit that includes this header has its own status word
// (a device variable is per module without relocatable device code), so
// each defines its reader with RNGX_BOUNDS_MODULE(name), listed in
// internal.h and read by rng_debug_bounds_status.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace rngx {

enum { kSiteGen = 10000, kSiteLfib = 20000, kSitePersist = 30000, kSiteDevice = 40000 };

#ifdef RNG_BOUNDS_CHECK
namespace {
__device__ int g_bounds_site;
}
__device__ __forceinline__ bool idx_ok(uint64_t i, uint64_t n, int site)
{
    if (i < n) return true;
    atomicCAS(&g_bounds_site, 0, site);
    return false;
}
// Shared-memory range [p, p + bytes) inside this block's dynamic shared memory.
__device__ __forceinline__ bool smem_ok(const void *p, const void *base, uint32_t bytes, int site)
{
    uint32_t dyn;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
    const uint64_t off = static_cast<uint64_t>(static_cast<const char *>(p) - static_cast<const char *>(base));
    return idx_ok(off + bytes - 1, dyn, site) && idx_ok(off, dyn, site);
}
#define RNGX_IDX_OK(i, n, site) ::rngx::idx_ok(static_cast<uint64_t>(i), static_cast<uint64_t>(n), (site))
#define RNGX_SMEM_OK(p, base, bytes, site) ::rngx::smem_ok((p), (base), (bytes), (site))
#define RNGX_BOUNDS_MODULE(name)                                                      \
    int bounds_site_##name(int *site, bool reset)                                     \
    {                                                                                 \
        cudaError_t e = cudaMemcpyFromSymbol(site, g_bounds_site, sizeof(int));       \
        if (e == cudaSuccess && reset) {                                              \
            const int zero = 0;                                                       \
            e = cudaMemcpyToSymbol(g_bounds_site, &zero, sizeof(int));                \
        }                                                                             \
        return e == cudaSuccess ? RNG_OK : ::rngx::cuda_fail(e, "bounds status");     \
    }
#else
#define RNGX_IDX_OK(i, n, site) true
#define RNGX_SMEM_OK(p, base, bytes, site) true
#define RNGX_BOUNDS_MODULE(name)                 \
    int bounds_site_##name(int *site, bool)      \
    {                                            \
        *site = 0;                               \
        return RNG_OK;                           \
    }
#endif

}  // namespace rngx
