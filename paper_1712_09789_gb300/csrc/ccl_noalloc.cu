// ccl_noalloc.cu -- ccl_label_noalloc(): the labelling pipeline with its
// scratch in a fixed, statically allocated device array instead of memory
// obtained from cudaMalloc.
//
// Who needs it: programs that may not allocate device memory once they are
// running -- for example a pipeline that has handed all of the GPU's memory to
// its own pool at start-up, or a latency-critical loop that must not call
// cudaMalloc/cudaFree because those calls can block and synchronise the whole
// device.  Such a caller still passes its own input and output buffers; only
// the scratch comes from this file.
//
// The array below is reserved on every GPU that loads the library, for as
// long as the process lives.  Its name is a host-side stand-in in host code,
// so its device address is fetched once per device with
// cudaGetSymbolAddress() while that device is current; the first call of the
// entry point on a device does that set-up, so that first call should happen
// before any stream capture.  All calls share the one array: calls whose work
// overlaps on the GPU (different streams, or different host threads) race on
// it and must be serialised by the caller.  No part of the array has to start
// at zero: every scratch entry the kernels read is written earlier in the
// same call, so what a previous call left behind is never used.
#include <cstddef>
#include <cstdint>
#include <mutex>

#include <cuda_runtime.h>

#include "../../include/ccl.h"
#include "ccl_internal.h"

namespace {

constexpr size_t kNoAllocScratchBytes = (size_t)64 << 20;  // 64 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_noalloc_mu;
void *g_noalloc_ptr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device, looked up once.
ccl_status noalloc_scratch(void **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CCL_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return CCL_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return CCL_ERR_CUDA;
        }
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return CCL_OK;
}

}  // namespace

extern "C" {

size_t ccl_noalloc_max_workspace_bytes(void) { return kNoAllocScratchBytes; }

ccl_status ccl_label_noalloc(const uint8_t *img, int H, int W, size_t pitch, int connectivity,
                             int32_t *labels, void *stream) {
    ccl_status st = ccl::check_image_args_api(img, H, W, pitch, connectivity, labels);
    if (st != CCL_OK || H == 0 || W == 0) return st;
    if (ccl::workspace_bytes(H, W) > kNoAllocScratchBytes) return CCL_ERR_UNSUPPORTED;
    void *ws = nullptr;
    if ((st = noalloc_scratch(&ws)) != CCL_OK) return st;
    if (ccl::launch_label(img, H, W, pitch, connectivity, labels, ws, static_cast<cudaStream_t>(stream),
                          ccl::iteration_cap_api()) != 0)
        return CCL_ERR_CUDA;
    return CCL_OK;
}

}  // extern "C"
