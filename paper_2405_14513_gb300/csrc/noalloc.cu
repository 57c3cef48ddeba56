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
#include <mutex>
#include <string>

#include "bisp.h"

namespace bisp {
int record_error(int code, const char *msg);
}

namespace {

constexpr size_t kStaticScratchBytes = size_t(64) << 20;   // 64 MiB
constexpr int kMaxDevices = 128;

// The workspace of estimator_estimate_static.  In host code its name is only
// a stand-in for the device symbol: its device address is looked up with
// cudaGetSymbolAddress (once per device) and passed to the kernels.
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_mu;
void *g_scratch_ptr[kMaxDevices] = {};

// Device address of g_static_scratch on the current device, looked up on the
// first call for that device.
int scratch_address(void **out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return bisp::record_error(BISP_CUDA_ERROR, (std::string("cudaGetDevice: ") + cudaGetErrorString(e)).c_str());
    if (dev < 0 || dev >= kMaxDevices) return bisp::record_error(BISP_INVALID_ARG, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p)
            return bisp::record_error(BISP_CUDA_ERROR,
                                      (std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e)).c_str());
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return BISP_OK;
}

}  // namespace

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
    void *scratch = nullptr;
    int st = scratch_address(&scratch);
    if (st) return st;
    // every workspace element the estimate reads is written earlier in the same
    // call, so nothing in the scratch has to start at zero
    return estimator_estimate(plan, delta, batch, scratch, B, stream);
}
