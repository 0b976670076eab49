// ccl_internal.h -- host-side interface between the C ABI and the kernels.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/ccl.h"

namespace ccl {

// One image of a launch.  Blocks of the image are the consecutive work items
// block0 .. block0 + nbx*nby - 1, in raster order.
constexpr unsigned kJobVecIn = 1;   // img and pitch are 16-byte aligned
constexpr unsigned kJobVecOut = 2;  // labels are 16-byte aligned and W % 4 == 0
struct Job {
    const uint8_t *img;
    int32_t *labels;
    unsigned long long pitch;
    int H, W;
    int nbx, nby;
    unsigned block0;
    unsigned flags;
    // raster position of the image's pixel (0, 0) within a larger image: 0
    // for a whole image, y0 * W for a strip whose first row is row y0
    unsigned key0;
    unsigned pad;
};

// Device header in front of a batch's job array.  The counters are the work
// queues of the kernels and must be zero when the launch starts.
struct JobHeader {
    unsigned njobs;
    unsigned total;       // work items (blocks) over all jobs
    unsigned counter[4];
    unsigned pad[2];
};

// Kernel argument: a batch (hdr and jobs in device memory, persistent CTAs)
// or, when hdr is null, the single job and its block count.
struct JobTable {
    JobHeader *hdr;
    const Job *jobs;
    Job single;
    unsigned total;
};

// Block shapes of a batch.  Lane-tile kernels (lane tiles across x down,
// lane tile rows): 0 = 16x16 of 32x4 (512x64 pixels, 256 threads), 1 = 8x16
// of 32x4 (256x64, 128 threads), 2 = 32x8 of 32x4 (1024x32, 256 threads),
// 3 = 16x8 of 32x8 (512x64, 128 threads).  Piece labeller: 4 = 512x64 (256
// threads), 5 = 256x32 (128 threads).
constexpr int kNumGeo = 6;
const char *geo_name(int geo);
size_t geo_blocks(int geo, int H, int W);
size_t geo_workspace_bytes(int geo, size_t blocks);
void geo_block_shape(int geo, int *bw, int *bh);

// Scratch bytes needed by launch_label() for an H x W image.
size_t workspace_bytes(int H, int W);

// Per-device set-up of a block shape (kernel attributes, occupancy); done
// implicitly by the launchers, and explicitly before a stream capture.
int prepare_geo(int geo);

// Enqueues the labelling of a batch: hdr/jobs are device copies (counters
// zero) for `capacity` blocks of scratch in `ws`.  Persistent grids.
int launch_jobs(int geo, int conn, JobHeader *hdr, const Job *jobs, void *ws, size_t capacity,
                cudaStream_t stream, int cap);

// Enqueues the whole labelling of one image on `stream`.  `ws` must hold
// workspace_bytes(H, W) bytes, 256-byte aligned.  `cap` <= 0 selects the
// default iteration caps.  `chain` lets the first kernel start while the
// kernel before it on the stream finishes (programmatic dependent launch;
// the piece labeller only): allowed only when that kernel may be the
// write-out of an earlier labelling whose scratch is not `ws` and whose
// labels do not overlap `img`.  Returns 0, or -1 when a launch failed.
int launch_label(const uint8_t *img, int H, int W, size_t pitch, int conn, int32_t *labels, void *ws,
                 cudaStream_t stream, int cap, bool chain = false);

// Strip sharding (ccl_strip.cu).  launch_label_phases() runs the kernels of
// launch_label() selected by `phases` on an image whose pixel (0, 0) has
// raster position key0 in the whole image: kPhaseLocalMerge = step 1 and the
// block merge, kPhaseWrite = the write-out (on the same `ws`, later).
constexpr int kPhaseLocalMerge = 1, kPhaseWrite = 2;
int launch_label_phases(const uint8_t *img, int H, int W, size_t pitch, int conn, uint32_t key0, int32_t *labels,
                        void *ws, cudaStream_t stream, int cap, int phases);
// Blocks of 512 x 64 pixels; each keeps a border record of kStripEdge slot
// numbers (top row, bottom row, left column, right column; kStripNoSlot for
// background) and kStripSlots union-find entries (key << 32 | parent).
constexpr int kStripBW = 512, kStripBH = 64, kStripSlots = 576, kStripEdge = 1152, kStripEdgeBottom = 512;
constexpr uint16_t kStripNoSlot = 0xFFFF;
struct ScratchView {
    uint16_t *edges;   // [blocks][kStripEdge]
    uint64_t *P;       // [blocks][kStripSlots]
    int32_t *nslots;   // [blocks]
    unsigned nbx, nby;
};
// Where launch_label() keeps those records in `ws` for an H x W image.
int label_scratch_view(int H, int W, int conn, void *ws, ScratchView *v);

// The coarse-labelling variants of Sec. 4.2 (mode 0 C2FL, 1 RC2FL, 2 CC2FL,
// 3 NC2FL) with counters, on 512x64 blocks; scratch of
// variant_workspace_bytes(H, W).  variant_counters reads the accumulated
// merges, find steps and CAS attempts of step 1 (and clears them if asked).
size_t variant_workspace_bytes(int H, int W);
int launch_label_variant(const uint8_t *img, int H, int W, size_t pitch, int conn, int mode, int32_t *labels,
                         void *ws, cudaStream_t stream, int cap);
int variant_counters(unsigned long long *out, bool reset);

// Component statistics (ccl_stats.cu): scratch bytes for an H x W image, and
// the enqueued pipeline; the component count lands in *count_dev and the
// number of pixels whose label names no root in *bad_dev (added to).
size_t stats_workspace_bytes(int H, int W);
int launch_stats(const int32_t *labels, int H, int W, ccl_component *out, int capacity, void *ws,
                 uint32_t *count_dev, int *bad_dev, cudaStream_t stream);

// 3D volumes (ccl_volume.cu): scratch bytes (face records) for a D x H x W
// volume, and the enqueued labelling (row stride pitch, slice stride
// H * pitch; connectivity 6 or 26).  Returns 0, or -1 when a launch failed.
size_t volume_workspace_bytes(int D, int H, int W);
int launch_volume(const uint8_t *img, int D, int H, int W, size_t pitch, int conn, int32_t *labels, void *ws,
                  cudaStream_t stream, int cap);

// Frees the batched runners (graphs, scratch, staging) of (dev, stream); the
// caller has waited for the stream.  Returns how many were freed.
int release_batched_stream(int dev, cudaStream_t stream);

// Reads the current device's error word and clears it.  Returns 0 or -1.
int read_and_clear_device_error(int *value);
int read_and_clear_volume_error(int *value);
int read_and_clear_strip_error(int *value);

// Argument checks and iteration cap of the C ABI, for entry points that live
// in other translation units (same rules as ccl_label()).
ccl_status check_image_args_api(const void *img, int H, int W, size_t pitch, int conn, const void *labels);
int iteration_cap_api();

// Benchmark timing of the kernels enqueued by launch_label().
// (kinds 0-2: the lane-tile kernels; 3 and 4: the piece labeller's step 1
// and step 3, whose step 2 is kind 1)
constexpr int kKindLocal = 0, kKindMerge = 1, kKindWrite = 2, kKindPieceLocal = 3, kKindPieceWrite = 4,
              kKindPieceCoop = 5;
constexpr int kKernelKinds = 6;
// a record of this kind closes the timing of one call
constexpr bool kind_closes_call(int k) { return k == kKindWrite || k == kKindPieceWrite || k == kKindPieceCoop; }
void timing_enable(bool on);
int timing_read(double *ms, long long *count, int n);
const char *kernel_kind_name(int k);

}  // namespace ccl
