// ols_noalloc.cu -- the adjoint with built-in scratch memory, for callers
// that cannot allocate device memory.
//
// ols_convolve_backward needs a scratch workspace (the ds overlap edges and
// the per-CTA dh spectra).  Some callers cannot provide one: real-time
// signal-processing pipelines that forbid any allocation once they are
// running (cudaMalloc can block and synchronise the device, which breaks
// their latency budget), and host programs that own every device allocation
// themselves and only lend the library the buffers of the operation.  This
// entry point serves them with a fixed scratch array that lives in the
// library's device image: every GPU that loads the library holds
// OLS_NOALLOC_SCRATCH_BYTES of it until the process exits.
//
// The array is a file-scope __device__ variable.  In host code its name is
// only a host-side stand-in, never a device address, so its address is
// looked up with cudaGetSymbolAddress once per device (with that device
// current) and that address is what the kernels receive.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "ols.h"
#include "ols_internal.h"

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[OLS_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void *g_scratch_ptr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device (set-up on the
// first call per device).  The address is cached for the life of the
// process: it belongs to the device's primary context, so a caller that
// destroys that context (cudaDeviceReset) must not call this entry point
// again in the same process.
int scratch_address(int dev, void **out) {
    if (dev < 0 || dev >= kMaxDevices) return OLS_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return OLS_ERR_CUDA;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return OLS_OK;
}

}  // namespace

extern "C" int ols_convolve_backward_noalloc(ols_plan_t plan, const float *s, int64_t Ns, const float *g,
                                             float *ds, float *dh, void *stream) {
    // the workspace entry point's checks first, so both report the same error
    int rc = ols::backward_validate(plan, s, Ns, g, ds, dh);
    if (rc != OLS_OK) return rc;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return OLS_ERR_CUDA;
    if (dev != plan->device) return OLS_ERR_INVALID;      // the plan's device must be current
    size_t need = 0;
    rc = ols_backward_workspace(plan, Ns, ds != nullptr, dh != nullptr, &need);
    if (rc != OLS_OK) return rc;
    if (need > (size_t)OLS_NOALLOC_SCRATCH_BYTES) return OLS_ERR_TOO_LARGE;
    void *scratch = nullptr;
    rc = scratch_address(dev, &scratch);
    if (rc != OLS_OK) return rc;
    // Nothing in the scratch needs to start at zero: the adjoint writes every
    // byte it later reads within the same call.
    return ols_convolve_backward(plan, s, Ns, g, ds, dh, scratch, (size_t)OLS_NOALLOC_SCRATCH_BYTES, stream);
}
