// ccl_stats.cu -- statistics of every component of a labelled image: area,
// bounding box and coordinate sums (centroid = sum / area), the size and
// location of each region that the paper gives as the use of labelling
// (Sec. 1).
//
// Canonical labels make the components easy to index: a pixel is its
// component's root when its label equals its own raster position plus one,
// and the roots in raster order are the components in label order.
//   k_stats_count       a bit per pixel (1 = root), and roots per chunk of
//                       8192 consecutive pixels
//   k_stats_scan        exclusive prefix over the chunk counts (one CTA)
//   k_stats_index       per 32-pixel word, the roots in the chunk's earlier
//                       words; component records initialised in label
//                       order.  The dense index of root p is then
//                       chunk prefix + word prefix + popcount below p (the
//                       bitmap and the prefixes are 3/16 B per pixel and
//                       stay in L2, where a 4 B/pixel index map did not)
//   k_stats_accumulate  tiles of 32 x 256 pixels: each pixel's component is
//                       looked up and its statistics folded into a shared-
//                       memory hash table, one global update per component
//                       and tile afterwards (the large components would
//                       otherwise meet in global atomics from every pixel);
//                       a component inside one tile gets plain stores
#include <climits>
#include <cstdint>

#include <cuda_runtime.h>

#include "ccl_internal.h"

namespace ccl {
namespace {

constexpr int kChunk = 8192;      // pixels per chunk (256 threads x 32)
constexpr int kStatThreads = 256;
constexpr int kTileH = 32, kTileW = 256;
constexpr int kHash = 1024;       // hash slots per tile
constexpr uint32_t kEmpty = 0xFFFFFFFFu;

__device__ __forceinline__ bool is_root(const int32_t *labels, long long p) {
    return labels[p] == (int32_t)(p + 1);
}

// Word j of chunk c holds pixels c * kChunk + 32 * j .. + 31 (a warp's step).
__global__ void __launch_bounds__(kStatThreads) k_stats_count(const int32_t *labels, long long n, uint32_t *bits,
                                                               uint32_t *counts) {
    __shared__ uint32_t warp_sum[kStatThreads / 32];
    const long long base = (long long)blockIdx.x * kChunk;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t c = 0;
    // all of a thread's loads first (independent, in flight together), then
    // the ballots
    constexpr int kSteps = kChunk / kStatThreads;
    int32_t v[kSteps];
#pragma unroll
    for (int i = 0; i < kSteps; ++i) {
        const long long p = base + (long long)(i * kStatThreads) + 32 * w + lane;
        v[i] = __ldg(labels + (p < n ? p : n - 1));  // unconditional: no branch between the loads
    }
#pragma unroll
    for (int i = 0; i < kSteps; ++i) {
        const long long q = base + (long long)(i * kStatThreads) + 32 * w;  // first pixel of the warp's word
        const long long p = q + lane;
        const unsigned m = __ballot_sync(0xFFFFFFFFu, p < n && v[i] == (int32_t)(p + 1));
        if (lane == 0 && q < n) bits[q >> 5] = m;
        c += (uint32_t)(lane == 0 ? __popc(m) : 0);
    }
    c = __reduce_add_sync(0xFFFFFFFFu, c);
    if ((threadIdx.x & 31) == 0) warp_sum[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t s = 0;
        for (int w = 0; w < kStatThreads / 32; ++w) s += warp_sum[w];
        counts[blockIdx.x] = s;
    }
}

// counts[0..nchunks) -> exclusive prefix in place; counts[nchunks] = total
__global__ void __launch_bounds__(1024) k_stats_scan(uint32_t *counts, int nchunks) {
    __shared__ uint32_t warp_sum[32];
    __shared__ uint32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int off = 0; off < nchunks; off += 1024) {
        const int i = off + (int)threadIdx.x;
        const uint32_t v = i < nchunks ? counts[i] : 0u;
        uint32_t incl = v;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t x = __shfl_up_sync(0xFFFFFFFFu, incl, d);
            if (lane >= d) incl += x;
        }
        if (lane == 31) warp_sum[w] = incl;
        __syncthreads();
        uint32_t before = carry;
        for (int k = 0; k < w; ++k) before += warp_sum[k];
        if (i < nchunks) counts[i] = before + incl - v;
        __syncthreads();
        if (threadIdx.x == 1023) carry = before + incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) counts[nchunks] = carry;
}

__global__ void __launch_bounds__(kStatThreads) k_stats_index(const uint32_t *bits, long long n,
                                                               const uint32_t *base, uint16_t *wpre,
                                                               ccl_component *out, int capacity) {
    __shared__ uint32_t warp_sum[kStatThreads / 32];
    static_assert(kChunk / 32 == kStatThreads, "one word of the chunk per thread");
    const long long word = (long long)blockIdx.x * (kChunk / 32) + threadIdx.x;
    const long long nwords = (n + 31) >> 5;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t m = word < nwords ? bits[word] : 0u;
    const uint32_t c = __popc(m);
    uint32_t incl = c;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t v = __shfl_up_sync(0xFFFFFFFFu, incl, d);
        if (lane >= d) incl += v;
    }
    if (lane == 31) warp_sum[w] = incl;
    __syncthreads();
    uint32_t before = incl - c;
    for (int k = 0; k < w; ++k) before += warp_sum[k];
    if (word < nwords) wpre[word] = (uint16_t)before;
    uint32_t idx = base[blockIdx.x] + before;
    for (uint32_t r = m; r; r &= r - 1, ++idx) {
        const long long p = word * 32 + (__ffs(r) - 1);
        if ((int)idx < capacity) {
            ccl_component cc;
            cc.label = (int32_t)(p + 1);
            cc.area = 0;
            cc.x0 = INT_MAX;
            cc.y0 = INT_MAX;
            cc.x1 = -1;
            cc.y1 = -1;
            cc.sum_x = 0;
            cc.sum_y = 0;
            out[idx] = cc;
        }
    }
}

// Dense index of pixel p when it is a root, else kEmpty.
__device__ __forceinline__ uint32_t root_index(const uint32_t *bits, const uint16_t *wpre, const uint32_t *base,
                                               long long p) {
    const uint32_t m = bits[p >> 5];
    const uint32_t b = 1u << (p & 31);
    if (!(m & b)) return kEmpty;
    return base[p / kChunk] + wpre[p >> 5] + __popc(m & (b - 1u));
}

// Per-tile statistics in tile coordinates (x - tx0, y - ty0): every field
// fits 32 bits (a tile has 8192 pixels of coordinates below 256), so all
// shared-memory updates are native 32-bit atomics.
struct StatSmem {
    uint32_t key[kHash];
    int32_t area[kHash], x0[kHash], y0[kHash], x1[kHash], y1[kHash];
    uint32_t sx[kHash], sy[kHash];
};

// Adds a tile's share of a component (tile coordinates from tx0, ty0) to its
// record.
__device__ __forceinline__ void fold_global(ccl_component *out, uint32_t k, int tx0, int ty0, int a, int x0, int y0,
                                            int x1, int y1, uint32_t sx, uint32_t sy) {
    ccl_component &c = out[k];
    atomicAdd(&c.area, a);
    atomicMin(&c.x0, tx0 + x0);
    atomicMin(&c.y0, ty0 + y0);
    atomicMax(&c.x1, tx0 + x1);
    atomicMax(&c.y1, ty0 + y1);
    atomicAdd(reinterpret_cast<unsigned long long *>(&c.sum_x), (unsigned long long)sx + (unsigned long long)a * tx0);
    atomicAdd(reinterpret_cast<unsigned long long *>(&c.sum_y), (unsigned long long)sy + (unsigned long long)a * ty0);
}

__global__ void __launch_bounds__(kStatThreads) k_stats_accumulate(const int32_t *labels, int H, int W,
                                                                    const uint32_t *bits, const uint16_t *wpre,
                                                                    const uint32_t *counts, int nchunks,
                                                                    ccl_component *out, int capacity, int *bad) {
    __shared__ StatSmem sm;
    for (int i = threadIdx.x; i < kHash; i += kStatThreads) {
        sm.key[i] = kEmpty;
        sm.area[i] = 0;
        sm.x0[i] = INT_MAX;
        sm.y0[i] = INT_MAX;
        sm.x1[i] = -1;
        sm.y1[i] = -1;
        sm.sx[i] = 0;
        sm.sy[i] = 0;
    }
    __syncthreads();
    const uint32_t ncomp = counts[nchunks];
    const uint32_t lim = ncomp < (uint32_t)capacity ? ncomp : (uint32_t)capacity;
    const long long n = (long long)H * W;
    const int tx0 = blockIdx.x * kTileW, ty0 = blockIdx.y * kTileH;
    const int lane = threadIdx.x & 31;
    int nbad = 0;
    // the lanes of a warp read 32 neighbouring pixels of a row; the lanes of
    // one component are folded first, so each component takes one
    // shared-memory update per warp step
    for (int i = threadIdx.x; i < kTileH * kTileW; i += kStatThreads) {
        const int rx = i % kTileW, ry = i / kTileW;
        const int x = tx0 + rx, y = ty0 + ry;
        uint32_t k = kEmpty;
        if (x < W && y < H) {
            const int32_t l = labels[(long long)y * W + x];
            if (l != 0) {
                // a label must name a root of the image (canonical labels);
                // anything else is counted and skipped
                const uint32_t r = (l < 0 || (long long)l > n) ? kEmpty : root_index(bits, wpre, counts, (long long)l - 1);
                if (r == kEmpty) {
                    ++nbad;
                } else {
                    k = r < lim ? r : kEmpty;
                }
            }
        }
        const unsigned peers = __match_any_sync(0xFFFFFFFFu, k);
        if (k == kEmpty) continue;
        // every lane of the group (all of `peers`) takes part in the
        // reductions; then the lowest lane updates for the whole group
        const int a = __popc(peers);
        const int gx0 = (int)__reduce_min_sync(peers, (unsigned)rx), gx1 = (int)__reduce_max_sync(peers, (unsigned)rx);
        const int gy0 = (int)__reduce_min_sync(peers, (unsigned)ry), gy1 = (int)__reduce_max_sync(peers, (unsigned)ry);
        const uint32_t gsx = __reduce_add_sync(peers, (unsigned)rx), gsy = __reduce_add_sync(peers, (unsigned)ry);
        if (lane != __ffs(peers) - 1) continue;
        uint32_t h = (k * 2654435761u) >> 22;  // 10-bit hash
        bool done = false;
        for (int probe = 0; probe < 16 && !done; ++probe, h = (h + 1) & (kHash - 1)) {
            uint32_t cur = sm.key[h];
            if (cur == kEmpty) cur = atomicCAS(&sm.key[h], kEmpty, k);
            if (cur == kEmpty || cur == k) {
                atomicAdd(&sm.area[h], a);
                atomicMin(&sm.x0[h], gx0);
                atomicMin(&sm.y0[h], gy0);
                atomicMax(&sm.x1[h], gx1);
                atomicMax(&sm.y1[h], gy1);
                atomicAdd(&sm.sx[h], gsx);
                atomicAdd(&sm.sy[h], gsy);
                done = true;
            }
        }
        if (!done) fold_global(out, k, tx0, ty0, a, gx0, gy0, gx1, gy1, gsx, gsy);
    }
    __syncthreads();
    // a component that reaches no tile edge shared with another tile lies in
    // this tile alone: its record is final and takes plain stores
    const int lastx = kTileW - 1, lasty = kTileH - 1;
    const bool right = tx0 + kTileW < W, below = ty0 + kTileH < H;
    for (int i = threadIdx.x; i < kHash; i += kStatThreads) {
        const uint32_t k = sm.key[i];
        if (k == kEmpty) continue;
        const int a = sm.area[i];
        const bool alone = !(sm.x0[i] == 0 && tx0 > 0) && !(sm.y0[i] == 0 && ty0 > 0) &&
                           !(sm.x1[i] == lastx && right) && !(sm.y1[i] == lasty && below);
        if (alone) {
            ccl_component &c = out[k];
            c.area = a;
            c.x0 = tx0 + sm.x0[i];
            c.y0 = ty0 + sm.y0[i];
            c.x1 = tx0 + sm.x1[i];
            c.y1 = ty0 + sm.y1[i];
            c.sum_x = (int64_t)sm.sx[i] + (int64_t)a * tx0;
            c.sum_y = (int64_t)sm.sy[i] + (int64_t)a * ty0;
        } else {
            fold_global(out, k, tx0, ty0, a, sm.x0[i], sm.y0[i], sm.x1[i], sm.y1[i], sm.sx[i], sm.sy[i]);
        }
    }
    if (nbad) atomicAdd(bad, nbad);
}

}  // namespace

// Scratch: the root bitmap (n / 8 bytes), the word prefixes (n / 16 bytes),
// the chunk counts.
namespace {
struct StatsLayout {
    size_t bits, wpre, counts, total;
};
StatsLayout stats_layout(long long n) {
    const long long nwords = (n + 31) / 32, nchunks = (n + kChunk - 1) / kChunk;
    StatsLayout l;
    size_t off = 0;
    l.bits = off;   off += ((size_t)nwords * 4 + 255) & ~(size_t)255;
    l.wpre = off;   off += ((size_t)nwords * 2 + 255) & ~(size_t)255;
    l.counts = off; off += ((size_t)(nchunks + 2) * 4 + 255) & ~(size_t)255;
    l.total = off;
    return l;
}
}  // namespace

size_t stats_workspace_bytes(int H, int W) { return stats_layout((long long)H * W).total; }

int launch_stats(const int32_t *labels, int H, int W, ccl_component *out, int capacity, void *ws,
                 uint32_t *count_dev, int *bad_dev, cudaStream_t stream) {
    const long long n = (long long)H * W;
    const int nchunks = (int)((n + kChunk - 1) / kChunk);
    const StatsLayout lay = stats_layout(n);
    char *w8 = static_cast<char *>(ws);
    uint32_t *bits = reinterpret_cast<uint32_t *>(w8 + lay.bits);
    uint16_t *wpre = reinterpret_cast<uint16_t *>(w8 + lay.wpre);
    uint32_t *counts = reinterpret_cast<uint32_t *>(w8 + lay.counts);
    k_stats_count<<<nchunks, kStatThreads, 0, stream>>>(labels, n, bits, counts);
    k_stats_scan<<<1, 1024, 0, stream>>>(counts, nchunks);
    k_stats_index<<<nchunks, kStatThreads, 0, stream>>>(bits, n, counts, wpre, out, capacity);
    const dim3 grid((W + kTileW - 1) / kTileW, (H + kTileH - 1) / kTileH);
    k_stats_accumulate<<<grid, kStatThreads, 0, stream>>>(labels, H, W, bits, wpre, counts, nchunks, out, capacity,
                                                         bad_dev);
    if (cudaMemcpyAsync(count_dev, counts + nchunks, sizeof(uint32_t), cudaMemcpyDeviceToDevice, stream) !=
        cudaSuccess)
        return -1;
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace ccl
