// ccl_internal.h -- host-side interface between the C ABI and the kernels.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace ccl {

// Scratch bytes needed by launch_label() for an H x W image.
size_t workspace_bytes(int H, int W);

// Enqueues the whole labelling of one image on `stream`.  `ws` must hold
// workspace_bytes(H, W) bytes, 256-byte aligned.  `cap` <= 0 selects the
// default iteration caps.  Returns 0, or -1 when a launch failed.
int launch_label(const uint8_t *img, int H, int W, size_t pitch, int conn, int32_t *labels, void *ws,
                 cudaStream_t stream, int cap);

// Reads the current device's error word and clears it.  Returns 0 or -1.
int read_and_clear_device_error(int *value);

// Benchmark timing of the kernels enqueued by launch_label().
constexpr int kKindLocal = 0, kKindMerge = 1, kKindFlatten = 2, kKindRelabel = 3;
constexpr int kKernelKinds = 4;
void timing_enable(bool on);
int timing_read(double *ms, long long *count, int n);
const char *kernel_kind_name(int k);

}  // namespace ccl
