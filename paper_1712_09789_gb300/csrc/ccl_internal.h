// ccl_internal.h -- host-side interface between the C ABI and the kernels.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/ccl.h"

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

// Argument checks and iteration cap of the C ABI, for entry points that live
// in other translation units (same rules as ccl_label()).
ccl_status check_image_args_api(const void *img, int H, int W, size_t pitch, int conn, const void *labels);
int iteration_cap_api();

// Benchmark timing of the kernels enqueued by launch_label().
constexpr int kKindLocal = 0, kKindMerge = 1, kKindRelabel = 2;
constexpr int kKernelKinds = 3;
void timing_enable(bool on);
int timing_read(double *ms, long long *count, int n);
const char *kernel_kind_name(int k);

}  // namespace ccl
