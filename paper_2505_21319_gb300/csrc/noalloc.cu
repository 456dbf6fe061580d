// efunc_forward_noalloc: the forward entry point for callers that cannot
// allocate device memory, with its scratch in a fixed array owned by this
// library instead of a caller-provided workspace.
#include <mutex>

#include "common.cuh"

namespace {

// Scratch of the no-allocation forward.  Every GPU that loads the library
// holds these bytes until the process exits.
constexpr size_t kNoAllocScratchBytes = (size_t)32 << 20;   // 32 MiB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_ptr[kMaxDevices];   // device address of g_noalloc_scratch, per device

// Device address of the scratch array on the current device.  The host-side
// name g_noalloc_scratch is only a stand-in for the symbol, never a device
// address, so the address is asked from the runtime once per device (with
// that device current) and cached.
cudaError_t noalloc_scratch(void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return cudaSuccess;
}

}  // namespace

namespace efunc {
efunc_status cuda_fail(cudaError_t e);   // records the error for efunc_last_cuda_error
}

extern "C" {

efunc_status efunc_forward_noalloc(const efunc_grid *grid, const float *params, const float *q, int64_t J,
                                   int32_t q_stride, float *O, float *lse, float *dOdq, efunc_stream_t stream)
{
    // the same host-side checks as efunc_forward, before touching the device
    if (!grid || grid->R < 1 || grid->R > efunc::kMaxR) return EFUNC_ERR_ARG;
    if (J < 0) return EFUNC_ERR_ARG;
    if (J == 0) return efunc_forward(grid, params, q, J, q_stride, O, lse, dOdq, nullptr, 0, stream);
    const size_t need = efunc_eval_workspace_bytes(grid, J);
    if (need == 0) return EFUNC_ERR_ARG;
    if (need > kNoAllocScratchBytes) return EFUNC_ERR_WORKSPACE;   // beyond the fixed scratch
    void *scratch = nullptr;
    const cudaError_t e = noalloc_scratch(&scratch);
    if (e != cudaSuccess) return efunc::cuda_fail(e);
    // efunc_forward clears the control block and histogram it reads before
    // use, so the previous call's contents of the shared array do not leak in
    return efunc_forward(grid, params, q, J, q_stride, O, lse, dOdq, scratch, kNoAllocScratchBytes, stream);
}

}  // extern "C"
