/*
 * ccl.h -- C ABI of the GB300 block-based connected-components labeller.
 *
 * Problem (Sec. 1 and the first paragraph of Sec. 3): given a 2D binary image
 * I(x,y) of H rows and W columns, give every connected foreground region one
 * ID.  A pixel's raster position is P(x,y) = x + y*W; its provisional label
 * is its own position and the root of an equivalence list is the element whose
 * label equals its own address (Sec. 3.1.1), with links always from the
 * larger label to the smaller (Sec. 3.1.3, Sec. 3.2).  The root is therefore
 * the smallest position of its component, and this library writes the
 * canonical labels
 *
 *     labels[y*W + x] = 0                                   if I(x,y) == 0
 *     labels[y*W + x] = 1 + min{ x' + y'*W : (x',y') in C }  if (x,y) in C
 *
 * for every connected component C.  The +1 frees 0 for the background.  Any
 * nonzero input byte is foreground.  Connectivity is 4 (the connectivity the
 * paper evaluates, Sec. 4.3) or 8.
 *
 * The method (Sec. 3): (1) each tile is labelled locally in on-chip memory by
 * coarse labelling -- row connection, column connection, unification of the
 * label-equivalence lists -- followed by a refinement that merges separated
 * sub-regions and an ID conversion to global positions (Kernel 1, Sec.
 * 3.1.1-3.1.4); (2) tiles are merged by analysing only the pixels on tile
 * boundaries (Kernel 2, Sec. 3.2, Eq. 1-2); (3) a root-find flattens the
 * global label map (Sec. 3.3).
 *
 * Conventions shared by every entry point
 *   - Memory: `img` is read-only, row stride `pitch` bytes (pitch >= W).
 *     `labels` is dense int32 with row stride W.  The two must not overlap.
 *     Device pointers unless the name says host.  The caller owns them.
 *   - Streams: `stream` is a cudaStream_t passed as void*; NULL is the legacy
 *     default stream.  Device entry points are asynchronous and ordered on
 *     `stream`; argument errors are reported synchronously and nothing is
 *     enqueued.  A device-side error (an iteration cap reached inside a
 *     union-find loop) is recorded in a per-device error word and reported by
 *     ccl_get_device_status().
 *   - Sizes: H, W >= 0; an image with H == 0 or W == 0 is a no-op that returns
 *     CCL_OK.  H*W must not exceed 2^31 - 2 (CCL_ERR_UNSUPPORTED otherwise),
 *     so that 1 + position fits an int32.
 *   - Threads: entry points may be called from several host threads; calls
 *     that share a stream are ordered by that stream.
 */
#ifndef CCL_H
#define CCL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CCL_OK = 0,
    CCL_ERR_INVALID_ARG = 1,
    CCL_ERR_UNSUPPORTED = 2,
    CCL_ERR_OUT_OF_MEMORY = 3,
    CCL_ERR_CUDA = 4,
    CCL_ERR_DEVICE_TIMEOUT = 5,
    CCL_ERR_BUSY = 6,
    CCL_ERR_NOT_FOUND = 7
} ccl_status;

/* Human-readable name of a status code (static string, never NULL). */
const char *ccl_status_string(int status);

/* Library ABI version: major * 10000 + minor * 100 + patch. */
int ccl_version(void);

/*
 * Label one image (Sec. 3, all three steps).
 *   img          device, u8 [H][pitch]; nonzero = foreground.
 *   H, W         rows and columns.
 *   pitch        input row stride in bytes, >= W.
 *   connectivity 4 or 8.
 *   labels       device, int32 [H][W] (row stride W), written in full.
 *   stream       cudaStream_t.
 * Uses a library-owned scratch buffer per (device, stream), grown on demand
 * (the growth is a cudaMalloc; call once outside stream capture before
 * capturing).  Returns CCL_ERR_INVALID_ARG for NULL pointers, negative sizes,
 * pitch < W, connectivity not in {4,8} or overlapping img/labels;
 * CCL_ERR_UNSUPPORTED when H*W > 2^31 - 2; CCL_ERR_OUT_OF_MEMORY when the
 * scratch cannot grow; CCL_ERR_CUDA when a launch fails.
 */
ccl_status ccl_label(const uint8_t *img, int H, int W, size_t pitch, int connectivity,
                     int32_t *labels, void *stream);

/*
 * Scratch bytes that ccl_label_ws() needs for an H x W image (independent of
 * the connectivity, which is accepted for symmetry).  Writes *bytes.
 */
ccl_status ccl_workspace_size(int H, int W, int connectivity, size_t *bytes);

/*
 * ccl_label() with caller-owned scratch: `workspace` is a device buffer of at
 * least ccl_workspace_size() bytes, 256-byte aligned, used only by the work
 * enqueued by this call (no other call may use it until that work is done).
 * Returns CCL_ERR_INVALID_ARG when it is NULL, misaligned or too small.
 */
ccl_status ccl_label_ws(const uint8_t *img, int H, int W, size_t pitch, int connectivity,
                        int32_t *labels, void *workspace, size_t workspace_bytes,
                        void *stream);

/*
 * Label an image held in HOST memory: copies it to library-owned device
 * buffers on `stream`, labels it, copies the labels back to `host_labels`
 * (int32 [H][W]) and waits for the stream before returning, so the labels
 * are ready on return.  Page-locked host buffers give the fastest copies.
 * Errors as ccl_label(), plus a device error found by the wait.
 */
ccl_status ccl_label_host(const uint8_t *host_img, int H, int W, size_t pitch,
                          int connectivity, int32_t *host_labels, void *stream);

/*
 * ccl_label_host() without the wait: the copy in, the labelling and the copy
 * out are only enqueued on `stream`, and the labels are in `host_labels`
 * once the stream has reached that point (cudaStreamSynchronize, an event,
 * or ccl_get_device_status()).  Both host buffers must stay valid and
 * untouched until then; they must be page-locked for the copies to run
 * asynchronously.  Each (device, stream) has its own staging buffers, so
 * images enqueued on several streams overlap their copies with one another's
 * labelling.  Errors as ccl_label() (argument errors synchronously, nothing
 * enqueued); device errors surface through ccl_get_device_status().
 */
ccl_status ccl_label_host_async(const uint8_t *host_img, int H, int W, size_t pitch,
                                int connectivity, int32_t *host_labels, void *stream);

/*
 * One image of a batch (device pointers; same rules as ccl_label()).
 */
typedef struct {
    const uint8_t *img;   /* u8 [H][pitch], nonzero = foreground */
    int32_t *labels;      /* int32 [H][W], row stride W */
    int H;
    int W;
    size_t pitch;         /* input row stride in bytes, >= W */
} ccl_image;

/*
 * Label n images of any sizes with one launch sequence (Sec. 3, all three
 * steps, for every image): persistent kernels take the blocks of all images
 * from a device work queue, and the sequence is replayed as a CUDA graph
 * held per (device, stream, connectivity, block shape).  `images` is a host
 * array of n entries; every entry is checked as in ccl_label() and an invalid
 * entry fails the whole call with nothing enqueued.  Entries with H or W = 0
 * are skipped.  Outputs of different entries must not overlap each other or
 * any input.  The block shape is $CCL_TILE if set (a ccl_tile_name()), else
 * the one tuned for this GPU, connectivity and mean image area; when none is
 * tuned yet the call runs ccl_autotune_batched() first, which labels the
 * batch several times (same result) and remembers the choice.  The library
 * owns per-stream device scratch and page-locked staging, grown on demand
 * (growth allocates; make one call outside stream capture first).
 * Asynchronous on `stream`.
 */
ccl_status ccl_label_batched(const ccl_image *images, int n, int connectivity, void *stream);

/* ccl_label_batched() with an explicit block shape (0 .. ccl_tile_count()-1). */
ccl_status ccl_label_batched_tile(const ccl_image *images, int n, int connectivity, int tile,
                                  void *stream);

/*
 * Times every block shape on this batch (the batch is labelled each time),
 * keeps the fastest for the batch's size class -- in memory and appended to
 * $CCL_AUTOTUNE_CACHE or ~/.cache/ccl_gb300/autotune.txt -- and writes it to
 * *tile (may be NULL).  Waits for `stream`.
 */
ccl_status ccl_autotune_batched(const ccl_image *images, int n, int connectivity, void *stream,
                                int *tile);

/* Block shape ccl_label_batched() would use for this batch; -1 if untuned. */
ccl_status ccl_batched_tile(const ccl_image *images, int n, int connectivity, int *tile);

/* Number of block shapes, and the name of one ("512x64": width x height, on
 * lane tiles of 32 x 4 pixels; "512x64x8": the same block on 32 x 8 lane
 * tiles). */
int ccl_tile_count(void);
const char *ccl_tile_name(int tile);

/* ---------------------------------------------------------------------------
 * Serving: a continuous-batching server for frames held in host memory.  The
 * paper labels single images; batching, admission and latency accounting are
 * properties of this library.
 *
 * A scheduler thread keeps submitted requests in arrival order and starts a
 * batch on an idle CUDA stream with as many requests from the front of the
 * queue as fit: at most max_batch per batch, at most max_slots on the device
 * at once, one connectivity per batch, and device memory carved from a
 * resident arena of hbm_budget_bytes -- each frame's image and labels plus
 * the batch's job table and labelling scratch (admission is by free arena
 * memory; the server uses no other device memory).  Requests that arrive
 * while others run are admitted as slots and memory free up.  A batch is:
 * frame copies in, the three labelling kernels over all blocks of all its
 * frames (persistent CTAs taking blocks from a device work counter), and
 * label copies out in increasing frame size; each request completes as soon
 * as its own labels are in host memory.  Batches on different streams
 * overlap on the device.
 */
typedef struct {
    int max_slots;            /* requests on the device at once, >= 1 */
    int n_streams;            /* CUDA streams, 1..16 */
    int max_batch;            /* requests per batch, >= 1 */
    int device;               /* CUDA device ordinal */
    size_t hbm_budget_bytes;  /* resident frame arena (inputs + labels), >= 1 MiB */
} ccl_server_config;

typedef struct {
    uint64_t submitted, completed, rejected;
    int in_flight, queued;
    uint64_t pixels;                    /* labelled pixels */
    size_t arena_bytes, arena_used_bytes;
    double p50_ms, p99_ms, max_ms, mean_ms;  /* submit -> labels in host memory */
    double gpixel_s;                    /* pixels / (last completion - first submit) */
    /* Stages, per request (each request of a batch counts its batch's
     * device stages once): queue = submit -> admitted into a batch (host
     * clock); h2d, label, d2h = the batch's frame copies in, its labelling
     * kernels and its label copies out (CUDA events on its stream). */
    double queue_p50_ms, queue_p99_ms;
    double h2d_p50_ms, h2d_p99_ms;
    double label_p50_ms, label_p99_ms;
    double d2h_p50_ms, d2h_p99_ms;
    uint64_t batches;                   /* batches retired */
    uint64_t multi_request_batches;     /* of those, batches of more than one request */
    uint64_t overlapped_batches;        /* batches whose device span (copy-in start to
                                           copy-out end) overlapped that of another
                                           batch retired before it */
    int max_batch_requests;             /* largest batch */
    int max_batches_in_flight;          /* most batches on the device at once */
} ccl_server_stats_t;

typedef struct ccl_server ccl_server;

/* Creates a server (allocates its arena and streams, starts its thread). */
ccl_status ccl_server_create(const ccl_server_config *config, ccl_server **server);

/*
 * Arena bytes one H x W frame needs when it is served alone (image, labels,
 * labelling scratch and job table).  A server refuses a frame larger than its
 * whole arena by this measure; size hbm_budget_bytes as a multiple of it for
 * the frames that should be on the device at once.
 */
ccl_status ccl_server_frame_bytes(int H, int W, size_t *bytes);

/*
 * Queues one frame: host_img u8 [H][pitch], host_labels int32 [H][W], both
 * owned by the caller and untouched by it until the request completes
 * (page-locked memory gives asynchronous copies).  Writes a ticket.
 * CCL_ERR_INVALID_ARG as ccl_label() (and for an empty frame),
 * CCL_ERR_UNSUPPORTED for a frame whose ccl_server_frame_bytes() exceeds the
 * whole arena.
 */
ccl_status ccl_server_submit(ccl_server *server, const uint8_t *host_img, int H, int W, size_t pitch,
                             int connectivity, int32_t *host_labels, uint64_t *ticket);

/*
 * Waits for a request (timeout_ms < 0: no limit).  Returns the request's
 * status once it completed and forgets the ticket; CCL_ERR_BUSY when the
 * timeout passed first (the ticket stays valid); CCL_ERR_NOT_FOUND for an
 * unknown or already collected ticket.
 */
ccl_status ccl_server_wait(ccl_server *server, uint64_t ticket, int timeout_ms);

/* Non-blocking: the request's status if complete, else CCL_ERR_BUSY. */
ccl_status ccl_server_poll(ccl_server *server, uint64_t ticket);

/* Counters and latency percentiles since creation or the last reset. */
ccl_status ccl_server_stats(ccl_server *server, ccl_server_stats_t *stats);
ccl_status ccl_server_reset_stats(ccl_server *server);

/*
 * Stops admitting, lets the batches on the device finish, fails requests that
 * never started with CCL_ERR_BUSY, and frees everything.  No call on the
 * server may follow, and none may be in progress.
 */
void ccl_server_destroy(ccl_server *server);

/*
 * ccl_label() for callers that may not allocate device memory while they run
 * -- e.g. a program that gave all of the GPU's memory to its own pool at
 * start-up, or a latency-critical loop that must not call cudaMalloc/cudaFree
 * because those can block and synchronise the whole device.  The paper has no
 * counterpart; this is a property of the library, not of the method.
 *
 * The caller still passes img and labels (same meaning as ccl_label()).  The
 * scratch is a fixed array of ccl_noalloc_max_workspace_bytes() bytes
 * (64 MiB) that every GPU loading the library reserves until the process
 * exits; this call allocates nothing.  Images whose ccl_workspace_size()
 * exceeds that limit (about 1.34 bytes per pixel, so about 50 million
 * pixels) are rejected with CCL_ERR_UNSUPPORTED and nothing is enqueued.  The first call on a device
 * looks up the array's device address, so make that first call before any
 * stream capture.  All calls share the array: calls whose work overlaps on the
 * GPU (other streams, other host threads) race on it and must be serialised by
 * the caller.  Leftover contents from earlier calls are never read.
 */
ccl_status ccl_label_noalloc(const uint8_t *img, int H, int W, size_t pitch, int connectivity,
                             int32_t *labels, void *stream);

/* Size in bytes of the fixed scratch array used by ccl_label_noalloc(). */
size_t ccl_noalloc_max_workspace_bytes(void);

/*
 * Frees what the library holds for `stream` on the current device: the
 * scratch and staging buffers of ccl_label(), ccl_label_host(),
 * ccl_label_host_async(), ccl_label_variant(), ccl_component_stats() and
 * ccl_label_3d(), and the graphs, scratch and staging of ccl_label_batched().
 * Waits for the stream first.  Call it before destroying a stream that was
 * given to those entry points; a later call on the stream allocates afresh.
 * The library has no other per-stream state.
 */
ccl_status ccl_release_stream(void *stream);

/*
 * Waits for `stream`, then reports and clears the current device's error
 * word: CCL_ERR_DEVICE_TIMEOUT when a union-find loop reached its iteration
 * cap since the last check (its outputs are then not valid), CCL_ERR_CUDA when
 * the wait itself failed, CCL_OK otherwise.
 */
ccl_status ccl_get_device_status(void *stream);

/*
 * Statistics of one component, as ccl_component_stats writes them: its
 * label, its pixel count, its inclusive bounding box (x0, y0)-(x1, y1) and
 * the sums of its pixels' coordinates (centroid = sum / area).  40 bytes.
 */
typedef struct {
    int32_t label;
    int32_t area;
    int32_t x0, y0, x1, y1;
    int64_t sum_x, sum_y;
} ccl_component;

/*
 * Size and location of every region of a labelled image (the uses of
 * labelling the paper names in Sec. 1).  `labels` is a device H x W int32
 * image of canonical labels, as ccl_label writes them (row stride W).  The
 * components are written to the device array `out` in increasing label
 * order, at most `capacity` of them; `*count` (host) receives the number of
 * components, which may exceed `capacity` (call again with more room).
 * Synchronous on `stream`; library-owned scratch of 4 bytes per pixel.
 * Errors: bad sizes or pointers -> CCL_ERR_INVALID_ARG; labels that are not
 * canonical (a label that names no root) -> CCL_ERR_INVALID_ARG after the
 * run, with *count set; H*W > 2^31-2 -> CCL_ERR_UNSUPPORTED.
 */
ccl_status ccl_component_stats(const int32_t *labels, int H, int W, ccl_component *out, int capacity, int *count,
                               void *stream);

/*
 * Coarse-labelling variants of Sec. 4.2, for the paper's comparison of the
 * coarse-to-fine strategy: variant 0 is the method (C2FL, what ccl_label
 * computes), 1 keeps the coarse labelling along rows only (RC2FL), 2 along
 * columns only (CC2FL), 3 drops it (NC2FL: the refinement does all merging).
 * All four write the same canonical labels.  Runs on 512x64 blocks with
 * library-owned scratch (as ccl_label).  When `counters` is not NULL the call
 * is synchronous and writes 3 counts of step 1 (Kernel 1) over the image:
 * [0] merges (list unions), [1] root-walk steps, [2] atomic CAS attempts.
 * Arguments as ccl_label; variant outside 0..3 -> CCL_ERR_INVALID_ARG.
 */
ccl_status ccl_label_variant(const uint8_t *img, int H, int W, size_t pitch, int connectivity, int variant,
                             int32_t *labels, unsigned long long *counters, void *stream);

/*
 * Label a 3D binary volume (Sec. 1 poses the task for 2D and 3D images; the
 * three steps of Sec. 3 are applied to blocks of 32 x 16 x 16 voxels).
 *   img          device, u8; voxel (x, y, z) at img[(z * H + y) * pitch + x]
 *                (row stride pitch, slice stride H * pitch); nonzero =
 *                foreground.
 *   D, H, W      slices, rows, columns.
 *   pitch        input row stride in bytes, >= W.
 *   connectivity 6 (face neighbours) or 26 (face, edge and corner neighbours).
 *   labels       device, int32 [D][H][W] dense, written in full: 0 for
 *                background, else 1 + the smallest raster position
 *                x + y*W + z*W*H of the voxel's component.
 *   stream       cudaStream_t; the call is stream-ordered and asynchronous.
 * Uses a library-owned scratch buffer per (device, stream) of about 4.3
 * bytes per voxel, grown on demand (a cudaMalloc; call once outside stream
 * capture before capturing).  Per block of 32 x 16 x 16 voxels it holds the
 * row masks, one 16-bit value per run or piece, the border-slot record of
 * every face voxel and the global union-find entries of the border slots,
 * each sized for the worst case; a call touches only the used part.  Returns CCL_ERR_INVALID_ARG for NULL pointers, negative sizes,
 * pitch < W, connectivity not in {6,26} or overlapping img/labels;
 * CCL_ERR_UNSUPPORTED when D*H*W > 2^31 - 2; CCL_ERR_OUT_OF_MEMORY when the
 * scratch cannot grow; CCL_ERR_CUDA when a launch fails.  Iteration caps are
 * reported by ccl_get_device_status().
 */
ccl_status ccl_label_3d(const uint8_t *img, int D, int H, int W, size_t pitch, int connectivity,
                        int32_t *labels, void *stream);

/*
 * Strip sharding of one image (Sec. 3.2's boundary analysis at the seams of
 * horizontal strips labelled separately, e.g. one strip per GPU).  Strip g is
 * rows [y0_g, y0_g + H_g) of an H_total x W image.  Each strip starts on a
 * multiple of 64 rows, and every strip but the last has a multiple of 64 rows
 * (the seams sit between block rows); H_total * W <= 2^31 - 2.  Per strip:
 *
 *   1. ccl_strip_begin(): step 1 and the block merge of the strip, with every
 *      key a raster position of the whole image, then its edge rows:
 *      edges[x] and edges[W + x] (device, uint32 [2][W]) = the smallest
 *      position, within the strip, of the component holding pixel x of the
 *      strip's first / last row; 0xFFFFFFFF for background.  `img` is the
 *      strip's first row (device, u8, row stride pitch), `workspace` as for
 *      ccl_label_ws() with the strip's H and W; it carries the strip's state
 *      until ccl_strip_finish().
 *   2. The caller gathers the edge rows of all strips in strip order into a
 *      host array of uint32 [strips][2][W] (an all-gather across GPUs).
 *   3. ccl_strip_resolve() (host only, no CUDA call): joins the keys of every
 *      pair of foreground pixels adjacent across a seam (the last row of strip
 *      g and the first row of strip g+1) and writes to `map` (host, uint32
 *      pairs) every key whose component reaches a smaller key through the
 *      seams, with the smallest such key, sorted by key.  *count = number of
 *      pairs; CCL_ERR_INVALID_ARG when it exceeds `capacity` (pairs) -- call
 *      with capacity 0 to size it.  At most 2 * (strips - 1) * W pairs.  Every
 *      strip computes the same map from the same gathered rows.
 *   4. ccl_strip_finish(): `map` (device copy of the pairs, `count` of them)
 *      is applied to the strip's union-find roots, then the write-out fills
 *      `labels` (device, int32 [H][W] of the strip) with the labels of the
 *      whole image: 1 + the smallest position of the component over all strips.
 *
 * Arguments of begin and finish for one strip must agree (H, W,
 * connectivity, y0, H_total, workspace).  Errors: CCL_ERR_INVALID_ARG for
 * NULL pointers, negative sizes, a strip off the 64-row grid, a strip outside
 * the image or a workspace that is NULL, misaligned or too small;
 * CCL_ERR_UNSUPPORTED when H_total * W > 2^31 - 2; CCL_ERR_CUDA when a launch
 * fails.  An iteration cap reached on the device is reported by
 * ccl_get_device_status().
 */
ccl_status ccl_strip_begin(const uint8_t *img, int H, int W, size_t pitch, int connectivity, int y0,
                           int H_total, void *workspace, size_t workspace_bytes, uint32_t *edges,
                           void *stream);
ccl_status ccl_strip_resolve(const uint32_t *edges, int strips, int W, int connectivity, uint32_t *map,
                             size_t capacity, size_t *count);
ccl_status ccl_strip_finish(int H, int W, int connectivity, int y0, int H_total, const uint32_t *map,
                            size_t count, int32_t *labels, void *workspace, size_t workspace_bytes,
                            void *stream);

/*
 * Test hook for failure detection: caps every find/union loop in the kernels
 * at `cap` iterations (cap <= 0 restores the default, which no valid input
 * can reach).  A low cap makes the loops give up, set the device error word
 * and return, so nothing spins.  Affects launches made after the call.
 */
void ccl_debug_set_iteration_cap(int cap);

/*
 * Benchmark hook.  While enabled, every call records CUDA events on its own
 * stream around each of its kernels and their durations accumulate per kind:
 * 0 block-local labelling, 1 block merge, 2 root-find and label write-out
 * (lane-tile kernels: 4-connected single images, batches, variants), 3 and 4
 * the piece labeller's local labelling and write-out (8-connected single
 * images; its merge is kind 1).  While enabled the kernels of a call run one
 * after another (no programmatic overlap).  Enabling or disabling waits for
 * pending events and clears the sums.
 */
void ccl_debug_kernel_timing(int enable);

/*
 * Waits for the recorded events and writes up to n per-kind sums in
 * milliseconds and launch counts.  Returns the number of kernel kinds.
 */
int ccl_debug_kernel_times(double *ms_sum, long long *counts, int n);

/* Kernel name of a kind (static string; "" when out of range). */
const char *ccl_debug_kernel_name(int kind);

#ifdef __cplusplus
}
#endif

#endif /* CCL_H */
