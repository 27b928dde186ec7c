// psa_noalloc.cu -- psa_sigma_min_static: the sigma_min grid evaluation for
// callers that cannot allocate device memory.
//
// Some callers have no way to obtain device scratch: code running inside a
// host that forbids cudaMalloc after start-up (a memory pool handed out once,
// a real-time loop, a plugin sandbox), or code that must not allocate while a
// stream is being captured. For them the scratch that psa_sigma_min takes as
// `workspace` lives here instead, in one file-scope device array of fixed size
// that the module carries for as long as the library is loaded.
//
// The host may not use the array's name as a device address (in host code it
// names a host-side stand-in), so every call looks the device address up with
// cudaGetSymbolAddress on the current device. The lookup allocates nothing, and
// doing it per call keeps the address right when the device's context is torn
// down and created again (cudaDeviceReset), which may load the module elsewhere.
#include <cuda_runtime.h>

#include "psa.h"
#include "psa_internal.h"

namespace {

__device__ __align__(256) unsigned char g_static_scratch[PSA_STATIC_SCRATCH_BYTES];

// Device address of g_static_scratch in the current device's context.
int static_scratch(void **out)
{
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) return PSA_ECUDA;
    *out = p;
    return PSA_OK;
}

}  // namespace

extern "C" int psa_sigma_min_static(const psa_band *A, const psa_grid *g, const double *eps, int32_t n_eps,
                                    const int32_t *idx, int64_t n_idx, double *sigma, uint32_t *mask,
                                    int8_t *status, int32_t *steps, const psa_lanczos_opts *opts, void *stream)
{
    // the arguments first (the codes of psa_sigma_min), then the size: the problem
    // must fit the fixed scratch with at least one warp (32 points) in flight
    const int arc = psa::check_sigma_min_args(A, g, eps, n_eps, idx, n_idx, sigma, opts);
    if (arc != PSA_OK) return arc;
    size_t need = 0;
    const int rc = psa_workspace_bytes(A, opts, 32, 0, &need);
    if (rc != PSA_OK) return rc;
    if (need > (size_t)PSA_STATIC_SCRATCH_BYTES) return PSA_ESTATIC;
    void *scratch = nullptr;
    const int rs = static_scratch(&scratch);
    if (rs != PSA_OK) return rs;
    return psa_sigma_min(A, g, eps, n_eps, idx, n_idx, sigma, mask, status, steps, opts, scratch,
                         (size_t)PSA_STATIC_SCRATCH_BYTES, stream);
}
