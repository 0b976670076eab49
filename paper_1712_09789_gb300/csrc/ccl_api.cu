// ccl_api.cu -- the C ABI declared in include/ccl.h: argument checks,
// library-owned scratch per (device, stream), host-buffer entry point and the
// device error word.
#include <cstdint>
#include <cstring>
#include <map>
#include <mutex>
#include <utility>

#include <cuda_runtime.h>

#include "../../include/ccl.h"
#include "ccl_internal.h"

namespace {

std::mutex g_mu;
int g_cap = 0;  // iteration cap for new launches; 0 = default

struct DevBuf {
    void *ptr = nullptr;
    size_t bytes = 0;
};

// scratch, and the host entry point's staging buffers, per (device, stream)
std::map<std::pair<int, cudaStream_t>, DevBuf> g_scratch;
std::map<std::pair<int, cudaStream_t>, DevBuf> g_host_img;
std::map<std::pair<int, cudaStream_t>, DevBuf> g_host_lab;
std::map<std::pair<int, cudaStream_t>, DevBuf> g_stats;  // component statistics scratch
std::map<std::pair<int, cudaStream_t>, DevBuf> g_volume; // workspace of the 3D labelling

// ccl_label() alternates between two halves of its scratch per (device,
// stream), so that a labelling's step 1 may start (chained) while the
// previous labelling's write-out, which reads the other half, still runs.
// The labels range of the previous call guards against an image that
// overlaps it.
struct Chain {
    int half = 0;
    uintptr_t lab0 = 0, lab1 = 0;
};
std::map<std::pair<int, cudaStream_t>, Chain> g_chain;

// Offset of the second half of a chained scratch buffer: the buffer's own
// middle, whatever image the call labels, so that calls of different sizes
// keep to their halves.
size_t split(const DevBuf &b) { return (b.bytes / 2) & ~(size_t)255; }

ccl_status grow(DevBuf &b, size_t need) {
    if (b.bytes >= need) return CCL_OK;
    if (b.ptr) {
        cudaFree(b.ptr);
        b.ptr = nullptr;
        b.bytes = 0;
    }
    // grow geometrically so that a sequence of larger images reallocates rarely
    size_t want = need + need / 4;
    if (cudaMalloc(&b.ptr, want) != cudaSuccess) {
        cudaGetLastError();
        if (cudaMalloc(&b.ptr, need) != cudaSuccess) {
            cudaGetLastError();
            return CCL_ERR_OUT_OF_MEMORY;
        }
        want = need;
    }
    b.bytes = want;
    return CCL_OK;
}

ccl_status check_image_args(const void *img, int H, int W, size_t pitch, int conn, const void *labels) {
    if (H < 0 || W < 0) return CCL_ERR_INVALID_ARG;
    if (conn != 4 && conn != 8) return CCL_ERR_INVALID_ARG;
    if (H == 0 || W == 0) return CCL_OK;
    if (!img || !labels) return CCL_ERR_INVALID_ARG;
    if (pitch < (size_t)W) return CCL_ERR_INVALID_ARG;
    if ((long long)H * (long long)W > 2147483646LL) return CCL_ERR_UNSUPPORTED;
    // the input span and the output span must not overlap
    const uintptr_t i0 = reinterpret_cast<uintptr_t>(img);
    const uintptr_t i1 = i0 + (size_t)(H - 1) * pitch + (size_t)W;
    const uintptr_t o0 = reinterpret_cast<uintptr_t>(labels);
    const uintptr_t o1 = o0 + (size_t)H * (size_t)W * sizeof(int32_t);
    if (i0 < o1 && o0 < i1) return CCL_ERR_INVALID_ARG;
    return CCL_OK;
}

int current_cap() {
    std::lock_guard<std::mutex> lk(g_mu);
    return g_cap;
}


// Copies a host image into the library's staging buffers of (device,
// stream), labels it and copies the labels back to host memory, all enqueued
// on `stream`.  Consecutive calls on one stream reuse the same staging
// buffers in stream order; calls on different streams have their own.
ccl_status enqueue_host(const uint8_t *host_img, int H, int W, size_t pitch, int connectivity,
                        int32_t *host_labels, void *stream) {
    ccl_status st = check_image_args(host_img, H, W, pitch, connectivity, host_labels);
    if (st != CCL_OK || H == 0 || W == 0) return st;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CCL_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t dpitch = ((size_t)W + 15) & ~(size_t)15;
    const size_t img_bytes = dpitch * (size_t)H;
    const size_t lab_bytes = (size_t)H * (size_t)W * sizeof(int32_t);
    const size_t need = ccl::workspace_bytes(H, W);
    // held until everything is enqueued (see ccl_label)
    std::lock_guard<std::mutex> lk(g_mu);
    DevBuf &b = g_scratch[{dev, s}];
    DevBuf &bi = g_host_img[{dev, s}];
    DevBuf &bl = g_host_lab[{dev, s}];
    // the scratch halves alternate with ccl_label's on the same stream
    const size_t half = (need + 255) & ~(size_t)255;
    if (b.bytes < 2 * half || bi.bytes < img_bytes || bl.bytes < lab_bytes) {
        if (cudaStreamSynchronize(s) != cudaSuccess) return CCL_ERR_CUDA;
        if ((st = grow(b, 2 * half)) != CCL_OK) return st;
        if ((st = grow(bi, img_bytes)) != CCL_OK) return st;
        if ((st = grow(bl, lab_bytes)) != CCL_OK) return st;
    }
    if (cudaMemcpy2DAsync(bi.ptr, dpitch, host_img, pitch, (size_t)W, (size_t)H, cudaMemcpyHostToDevice, s) !=
        cudaSuccess)
        return CCL_ERR_CUDA;
    Chain &c = g_chain[{dev, s}];
    if (ccl::launch_label(static_cast<const uint8_t *>(bi.ptr), H, W, dpitch, connectivity,
                          static_cast<int32_t *>(bl.ptr), static_cast<char *>(b.ptr) + (c.half ? split(b) : 0), s,
                          g_cap) != 0)
        return CCL_ERR_CUDA;
    c.half ^= 1;
    c.lab0 = reinterpret_cast<uintptr_t>(bl.ptr);
    c.lab1 = c.lab0 + lab_bytes;
    if (cudaMemcpyAsync(host_labels, bl.ptr, lab_bytes, cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return CCL_ERR_CUDA;
    return CCL_OK;
}

}  // namespace

namespace ccl {

ccl_status check_image_args_api(const void *img, int H, int W, size_t pitch, int conn, const void *labels) {
    return check_image_args(img, H, W, pitch, conn, labels);
}

int iteration_cap_api() { return current_cap(); }

}  // namespace ccl

extern "C" {

const char *ccl_status_string(int status) {
    switch (status) {
        case CCL_OK: return "CCL_OK";
        case CCL_ERR_INVALID_ARG: return "CCL_ERR_INVALID_ARG";
        case CCL_ERR_UNSUPPORTED: return "CCL_ERR_UNSUPPORTED";
        case CCL_ERR_OUT_OF_MEMORY: return "CCL_ERR_OUT_OF_MEMORY";
        case CCL_ERR_CUDA: return "CCL_ERR_CUDA";
        case CCL_ERR_DEVICE_TIMEOUT: return "CCL_ERR_DEVICE_TIMEOUT";
        case CCL_ERR_BUSY: return "CCL_ERR_BUSY";
        case CCL_ERR_NOT_FOUND: return "CCL_ERR_NOT_FOUND";
        default: return "CCL_ERR_UNKNOWN";
    }
}

int ccl_version(void) { return 100; }

void ccl_debug_set_iteration_cap(int cap) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_cap = cap > 0 ? cap : 0;
}

ccl_status ccl_workspace_size(int H, int W, int connectivity, size_t *bytes) {
    if (!bytes || H < 0 || W < 0 || (connectivity != 4 && connectivity != 8)) return CCL_ERR_INVALID_ARG;
    if ((long long)H * (long long)W > 2147483646LL) return CCL_ERR_UNSUPPORTED;
    *bytes = (H == 0 || W == 0) ? 0 : ccl::workspace_bytes(H, W);
    return CCL_OK;
}

ccl_status ccl_label_ws(const uint8_t *img, int H, int W, size_t pitch, int connectivity, int32_t *labels,
                        void *workspace, size_t workspace_bytes, void *stream) {
    ccl_status st = check_image_args(img, H, W, pitch, connectivity, labels);
    if (st != CCL_OK || H == 0 || W == 0) return st;
    if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255) != 0 ||
        workspace_bytes < ccl::workspace_bytes(H, W))
        return CCL_ERR_INVALID_ARG;
    if (ccl::launch_label(img, H, W, pitch, connectivity, labels, workspace,
                          static_cast<cudaStream_t>(stream), current_cap()) != 0)
        return CCL_ERR_CUDA;
    return CCL_OK;
}

ccl_status ccl_label(const uint8_t *img, int H, int W, size_t pitch, int connectivity, int32_t *labels,
                     void *stream) {
    ccl_status st = check_image_args(img, H, W, pitch, connectivity, labels);
    if (st != CCL_OK || H == 0 || W == 0) return st;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CCL_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t need = ccl::workspace_bytes(H, W);
    // The lock is held until the launches are enqueued: another host thread
    // on the same stream that needs a larger buffer would otherwise free this
    // one after its stream wait but before this call's kernels are on the
    // stream.
    std::lock_guard<std::mutex> lk(g_mu);
    DevBuf &b = g_scratch[{dev, s}];
    const size_t half = (need + 255) & ~(size_t)255;
    if (b.bytes < 2 * half) {
        // the old buffer may still be in use by earlier work on this stream
        if (b.ptr && cudaStreamSynchronize(s) != cudaSuccess) return CCL_ERR_CUDA;
        st = grow(b, 2 * half);
        if (st != CCL_OK) return st;
    }
    Chain &c = g_chain[{dev, s}];
    const uintptr_t i0 = reinterpret_cast<uintptr_t>(img), i1 = i0 + (size_t)(H - 1) * pitch + (size_t)W;
    const bool chain = !(i0 < c.lab1 && c.lab0 < i1);
    void *ws = static_cast<char *>(b.ptr) + (c.half ? split(b) : 0);
    if (ccl::launch_label(img, H, W, pitch, connectivity, labels, ws, s, g_cap, chain) != 0) return CCL_ERR_CUDA;
    c.half ^= 1;
    c.lab0 = reinterpret_cast<uintptr_t>(labels);
    c.lab1 = c.lab0 + (size_t)H * (size_t)W * sizeof(int32_t);
    return CCL_OK;
}

ccl_status ccl_label_variant(const uint8_t *img, int H, int W, size_t pitch, int connectivity, int variant,
                             int32_t *labels, unsigned long long *counters, void *stream) {
    if (variant < 0 || variant > 3) return CCL_ERR_INVALID_ARG;
    ccl_status st = check_image_args(img, H, W, pitch, connectivity, labels);
    if (st != CCL_OK) return st;
    if (counters) {
        unsigned long long tmp[3];
        if (cudaDeviceSynchronize() != cudaSuccess || ccl::variant_counters(tmp, true) != 0) return CCL_ERR_CUDA;
    }
    if (H > 0 && W > 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) return CCL_ERR_CUDA;
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        const size_t need = ccl::variant_workspace_bytes(H, W);
        // held until the launches are enqueued (see ccl_label)
        std::lock_guard<std::mutex> lk(g_mu);
        DevBuf &b = g_scratch[{dev, s}];
        if (b.bytes < need) {
            if (b.ptr && cudaStreamSynchronize(s) != cudaSuccess) return CCL_ERR_CUDA;
            st = grow(b, need);
            if (st != CCL_OK) return st;
        }
        if (ccl::launch_label_variant(img, H, W, pitch, connectivity, variant, labels, b.ptr, s, g_cap) != 0)
            return CCL_ERR_CUDA;
    }
    if (counters) {
        if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess ||
            ccl::variant_counters(counters, false) != 0)
            return CCL_ERR_CUDA;
    }
    return CCL_OK;
}

ccl_status ccl_component_stats(const int32_t *labels, int H, int W, ccl_component *out, int capacity, int *count,
                               void *stream) {
    if (H < 0 || W < 0 || !count || capacity < 0 || (capacity > 0 && !out)) return CCL_ERR_INVALID_ARG;
    if ((long long)H * (long long)W > 2147483646LL) return CCL_ERR_UNSUPPORTED;
    *count = 0;
    if (H == 0 || W == 0) return CCL_OK;
    if (!labels) return CCL_ERR_INVALID_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CCL_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t ws_bytes = (ccl::stats_workspace_bytes(H, W) + 255) & ~(size_t)255;
    uint32_t host[2] = {0, 0};
    {
        // held until the call's work is done: the count is read back from
        // the shared scratch (see ccl_label)
        std::lock_guard<std::mutex> lk(g_mu);
        DevBuf &b = g_stats[{dev, s}];
        if (b.bytes < ws_bytes + 256) {
            if (b.ptr && cudaStreamSynchronize(s) != cudaSuccess) return CCL_ERR_CUDA;
            const ccl_status st = grow(b, ws_bytes + 256);
            if (st != CCL_OK) return st;
        }
        void *ws = b.ptr;
        // the last 256 bytes hold the component count and the count of bad pixels
        uint32_t *tail = reinterpret_cast<uint32_t *>(static_cast<char *>(ws) + ws_bytes);
        if (cudaMemsetAsync(tail, 0, 8, s) != cudaSuccess) return CCL_ERR_CUDA;
        if (ccl::launch_stats(labels, H, W, out, capacity, ws, tail, reinterpret_cast<int *>(tail + 1), s) != 0)
            return CCL_ERR_CUDA;
        if (cudaMemcpyAsync(host, tail, sizeof(host), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return CCL_ERR_CUDA;
    }
    *count = (int)host[0];
    return host[1] ? CCL_ERR_INVALID_ARG : CCL_OK;
}

ccl_status ccl_label_host(const uint8_t *host_img, int H, int W, size_t pitch, int connectivity,
                          int32_t *host_labels, void *stream) {
    ccl_status st = enqueue_host(host_img, H, W, pitch, connectivity, host_labels, stream);
    if (st != CCL_OK || H == 0 || W == 0) return st;
    return ccl_get_device_status(stream);
}

ccl_status ccl_label_host_async(const uint8_t *host_img, int H, int W, size_t pitch, int connectivity,
                                int32_t *host_labels, void *stream) {
    return enqueue_host(host_img, H, W, pitch, connectivity, host_labels, stream);
}

ccl_status ccl_release_stream(void *stream) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CCL_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaStreamSynchronize(s) != cudaSuccess) return CCL_ERR_CUDA;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        for (auto *m : {&g_scratch, &g_host_img, &g_host_lab, &g_stats, &g_volume}) {
            auto it = m->find({dev, s});
            if (it == m->end()) continue;
            if (it->second.ptr) cudaFree(it->second.ptr);
            m->erase(it);
        }
        g_chain.erase({dev, s});
    }
    ccl::release_batched_stream(dev, s);
    return CCL_OK;
}

void ccl_debug_kernel_timing(int enable) { ccl::timing_enable(enable != 0); }

int ccl_debug_kernel_times(double *ms_sum, long long *counts, int n) {
    if (!ms_sum || !counts || n < 0) return ccl::kKernelKinds;
    return ccl::timing_read(ms_sum, counts, n);
}

const char *ccl_debug_kernel_name(int kind) { return ccl::kernel_kind_name(kind); }

ccl_status ccl_get_device_status(void *stream) {
    if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess) return CCL_ERR_CUDA;
    int v = 0, vv = 0, vs = 0;
    if (ccl::read_and_clear_device_error(&v) != 0) return CCL_ERR_CUDA;
    if (ccl::read_and_clear_volume_error(&vv) != 0) return CCL_ERR_CUDA;
    if (ccl::read_and_clear_strip_error(&vs) != 0) return CCL_ERR_CUDA;
    return (v | vv | vs) ? CCL_ERR_DEVICE_TIMEOUT : CCL_OK;
}

ccl_status ccl_label_3d(const uint8_t *img, int D, int H, int W, size_t pitch, int connectivity, int32_t *labels,
                        void *stream) {
    if (D < 0 || H < 0 || W < 0) return CCL_ERR_INVALID_ARG;
    if (connectivity != 6 && connectivity != 26) return CCL_ERR_INVALID_ARG;
    if (D == 0 || H == 0 || W == 0) return CCL_OK;
    if (!img || !labels) return CCL_ERR_INVALID_ARG;
    if (pitch < (size_t)W) return CCL_ERR_INVALID_ARG;
    const long long n = (long long)D * (long long)H * (long long)W;
    if (n > 2147483646LL) return CCL_ERR_UNSUPPORTED;
    // the input span and the output span must not overlap
    const uintptr_t i0 = reinterpret_cast<uintptr_t>(img);
    const uintptr_t i1 = i0 + (size_t)((long long)D * H - 1) * pitch + (size_t)W;
    const uintptr_t o0 = reinterpret_cast<uintptr_t>(labels);
    const uintptr_t o1 = o0 + (size_t)n * sizeof(int32_t);
    if (i0 < o1 && o0 < i1) return CCL_ERR_INVALID_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CCL_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t need = ccl::volume_workspace_bytes(D, H, W);
    // held until the launches are enqueued (see ccl_label)
    std::lock_guard<std::mutex> lk(g_mu);
    DevBuf &b = g_volume[{dev, s}];
    if (b.bytes < need) {
        if (b.ptr && cudaStreamSynchronize(s) != cudaSuccess) return CCL_ERR_CUDA;
        const ccl_status st = grow(b, need);
        if (st != CCL_OK) return st;
    }
    if (ccl::launch_volume(img, D, H, W, pitch, connectivity, labels, b.ptr, s, g_cap) != 0)
        return CCL_ERR_CUDA;
    return CCL_OK;
}

}  // extern "C"
