// noalloc.cu -- estimator_estimate_static: the estimate of estimator_estimate
// with its workspace in a file-scope device array instead of caller memory.
//
// Some callers cannot allocate device memory at the point where they run the
// estimate: code under a memory manager that owns the whole device heap (a
// framework caching allocator, an MPI or serving runtime that hands out fixed
// pools) and must not see stray allocations, or plugins that are given a
// device and a stream but no allocator.  For plans small enough, this entry
// point needs nothing from the caller but the input field and the output
// array.
//
// The scratch array below is part of the library's device image: every GPU on
// which the library's module is loaded holds its kStaticScratchBytes until the
// process exits.
#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "bisp.h"
#include "kernels.cuh"

namespace bisp {
int record_error(int code, const char *msg);
}

namespace {

constexpr size_t kStaticScratchBytes = size_t(64) << 20;   // 64 MiB

// The workspace of estimator_estimate_static.  In host code its name is only
// a stand-in for the device symbol: its device address is looked up with
// cudaGetSymbolAddress, on the device that is current, and passed to the
// kernels.
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

int cuda_fail(const char *what, cudaError_t e)
{
    return bisp::record_error(BISP_CUDA_ERROR, (std::string(what) + ": " + cudaGetErrorString(e)).c_str());
}

}  // namespace

// Device address of g_static_scratch on the current device.  Looked up on
// every call (cheap once the module is loaded), so nothing stale survives a
// cudaDeviceReset; the first lookup on a device loads the library's module
// there.
int bisp::static_scratch_address(void **out)
{
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p) return cuda_fail("cudaGetSymbolAddress", e);
    *out = p;
    return BISP_OK;
}

extern "C" size_t estimator_static_scratch_bytes(void) { return kStaticScratchBytes; }

extern "C" int estimator_estimate_static(bisp_plan *plan, const void *delta, int batch, double *B, void *stream)
{
    if (!plan || !delta || !B) return bisp::record_error(BISP_INVALID_ARG, "NULL argument");
    const size_t need = estimator_workspace_bytes(plan, batch);
    if (need == 0) return bisp::record_error(BISP_INVALID_ARG, "batch out of range for this plan");
    if (need > kStaticScratchBytes) {
        std::string msg = "plan needs " + std::to_string(need) + " bytes of workspace; the static scratch of "
                          "estimator_estimate_static holds " + std::to_string(kStaticScratchBytes) +
                          " (use estimator_estimate with a caller workspace)";
        return bisp::record_error(BISP_INVALID_ARG, msg.c_str());
    }
    // the array used is the current device's: the plan and the stream must
    // belong to that device too
    int dev = -1, sdev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail("cudaGetDevice", e);
    e = cudaStreamGetDevice(static_cast<cudaStream_t>(stream), &sdev);
    if (e != cudaSuccess) return cuda_fail("cudaStreamGetDevice", e);
    if (sdev != dev || bisp::plan_device(plan) != dev)
        return bisp::record_error(BISP_INVALID_ARG, "the plan, the stream and the current device differ");
    void *scratch = nullptr;
    const int st = bisp::static_scratch_address(&scratch);
    if (st) return st;
    // every workspace element the estimate reads is written earlier in the
    // same call (the wait status too: it is cleared first), so nothing in the
    // scratch has to start at zero
    return estimator_estimate(plan, delta, batch, scratch, B, stream);
}
