// ccl_kernels.cu -- the three steps of the block-based labeller as sm_103a
// kernels, and the launcher that enqueues them on a stream.
//
//   k_local_border  step 1, Kernel 1 (Sec. 3.1): tile-local coarse labelling
//                   and refinement in shared memory; writes only what the
//                   block merge needs -- the tile's border record (which
//                   border-component every border pixel belongs to) and one
//                   union-find entry per border-touching component.
//   k_block_merge   step 2, Kernel 2 (Sec. 3.2): only pixel pairs that
//                   straddle a tile edge are examined; matching foreground
//                   pairs merge their components in the global union-find.
//   k_flatten       step 3, first half (Sec. 3.3): root-find for every
//                   border component, so each entry names its final root.
//   k_relabel       step 3, second half: recomputes the tile-local labelling
//                   from the image (instead of storing it), looks up the
//                   final key of each border component and writes
//                   1 + key for every foreground pixel, 0 for background.
//
// HBM traffic per pixel: 1 B image read in k_local_border, 1 B image read
// (often an L2 hit) and 4 B label write in k_relabel, plus the border records
// (2 B per border pixel) and union-find entries (8 B per border component).
#include <cstdint>
#include <deque>
#include <mutex>
#include <vector>

#include <cuda_runtime.h>

#include "ccl_internal.h"
#include "ccl_tile.cuh"

namespace ccl {

__device__ int g_device_error = 0;

struct ImageArgs {
    const uint8_t *img;
    int32_t *labels;
    size_t pitch;
    int H, W;
    int ntx, nty;
    bool vec_ok;       // img and pitch 16-byte aligned
    bool out_vec_ok;   // labels 16-byte aligned and W % 4 == 0
};

struct Scratch {
    uint16_t *edges;   // [ntiles][kEdge]
    uint64_t *P;       // [ntiles][kSlots]
    int32_t *nslots;   // [ntiles]
};

__device__ __forceinline__ void clear_tile_state(TileSmem &sm) {
    for (int i = threadIdx.x; i < kNodes / 32; i += kThreads) sm.border[i] = 0u;
    if (threadIdx.x == 0) sm.err = 0;
}

__device__ __forceinline__ void report(int err) {
    if (err) atomicOr(&g_device_error, err);
}

// ---------------------------------------------------------------------------
template <bool kConn8>
__global__ void __launch_bounds__(kThreads) k_local_border(ImageArgs a, Scratch s, int cap) {
    __shared__ TileSmem sm;
    const int t = blockIdx.x;
    const int tx = t % a.ntx, ty = t / a.ntx;
    const int x0 = tx * kTileW, y0 = ty * kTileH;
    clear_tile_state(sm);

    uint32_t m, S;
    label_tile<kConn8>(sm, a.img, a.H, a.W, a.pitch, a.vec_ok, x0, y0, cap, m, S);
    number_border_roots(sm);

    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint16_t *E = s.edges + (size_t)t * kEdge;
    // border record: slot of the pixel's component, or kBg
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int rr = k ? kTileH - 1 : 0;
        const uint32_t mm = sm.rowm[w][rr];
        uint16_t v = kBg;
        if ((mm >> lane) & 1u) {
            const int a0 = hibit(sm.runs[w][rr] & upto(lane));
            v = (uint16_t)border_slot(sm, sm.parent[swz(rr * kTileW + kSubW * w + a0)]);
        }
        E[(k ? kEdgeBottom : kEdgeTop) + kSubW * w + lane] = v;
    }
    if (w == 0) {
        const uint16_t v = (m & 1u) ? (uint16_t)border_slot(sm, sm.parent[swz(lane * kTileW)]) : kBg;
        E[kEdgeLeft + lane] = v;
    }
    if (w == kWarps - 1) {
        uint16_t v = kBg;
        if (m >> 31) v = (uint16_t)border_slot(sm, sm.parent[swz(lane * kTileW + kSubW * w + hibit(S))]);
        E[kEdgeRight + lane] = v;
    }
    // one union-find entry per border component: a root keyed by its
    // minimum global raster position (ID conversion, Sec. 3.1.4)
    {
        const int word = threadIdx.x;  // kNodes / 32 == kThreads
        uint32_t bits = sm.border[word];
        int slot = (int)sm.prefix[word];
        const uint32_t base = (uint32_t)t * kSlots;
        for (; bits; bits &= bits - 1, ++slot) {
            const int node = word * 32 + __ffs(bits) - 1;
            s.P[base + slot] = pack_slot(node_key(node, x0, y0, a.W), base + (uint32_t)slot);
        }
    }
    if (threadIdx.x == 0) {
        s.nslots[t] = sm.nslots;
        report(sm.err);
    }
}

// ---------------------------------------------------------------------------
// Each tile examines the pixel pairs across its top edge, its left edge and
// (8-connectivity) its two upper corners; the right, bottom and lower corners
// belong to the neighbouring tiles.  Thread j takes top-edge column j and,
// for j < kTileH, left-edge row j.  A pair that repeats the pair of the
// neighbouring thread is skipped.
template <bool kConn8>
__global__ void __launch_bounds__(kThreads) k_block_merge(Scratch s, int ntx, int nty, int cap) {
    const int t = blockIdx.x;
    const int tx = t % ntx, ty = t / ntx;
    const int j = threadIdx.x;
    const uint16_t *E = s.edges + (size_t)t * kEdge;
    const uint32_t base = (uint32_t)t * kSlots;
    int err = 0;

    if (ty > 0) {
        const int tu = t - ntx;
        const uint16_t *Eu = s.edges + (size_t)tu * kEdge;
        const uint32_t ubase = (uint32_t)tu * kSlots;
        const uint16_t a = E[kEdgeTop + j];
        if (a != kBg) {
            const uint16_t aL = j > 0 ? E[kEdgeTop + j - 1] : kBg;
            const uint16_t aR = j + 1 < kTileW ? E[kEdgeTop + j + 1] : kBg;
            const uint16_t b = Eu[kEdgeBottom + j];
            const uint16_t bL = j > 0 ? Eu[kEdgeBottom + j - 1] : kBg;
            if (b != kBg && !(aL == a && bL == b)) union_global(s.P, base + a, ubase + b, cap, err);
            if (kConn8) {
                // up-left: same pair as the left neighbour's vertical pair when aL == a
                if (j > 0) {
                    if (bL != kBg && aL != a) union_global(s.P, base + a, ubase + bL, cap, err);
                } else if (tx > 0) {
                    const uint16_t c = s.edges[(size_t)(tu - 1) * kEdge + kEdgeBottom + kTileW - 1];
                    if (c != kBg) union_global(s.P, base + a, (uint32_t)(tu - 1) * kSlots + c, cap, err);
                }
                // up-right: same pair as the right neighbour's vertical pair when aR == a
                if (j + 1 < kTileW) {
                    const uint16_t bR = Eu[kEdgeBottom + j + 1];
                    if (bR != kBg && aR != a) union_global(s.P, base + a, ubase + bR, cap, err);
                } else if (tx + 1 < ntx) {
                    const uint16_t c = s.edges[(size_t)(tu + 1) * kEdge + kEdgeBottom + 0];
                    if (c != kBg) union_global(s.P, base + a, (uint32_t)(tu + 1) * kSlots + c, cap, err);
                }
            }
        }
    }
    if (tx > 0 && j < kTileH) {
        const int tl = t - 1;
        const uint16_t *El = s.edges + (size_t)tl * kEdge;
        const uint32_t lbase = (uint32_t)tl * kSlots;
        const uint16_t a = E[kEdgeLeft + j];
        if (a != kBg) {
            const uint16_t aU = j > 0 ? E[kEdgeLeft + j - 1] : kBg;
            const uint16_t aD = j + 1 < kTileH ? E[kEdgeLeft + j + 1] : kBg;
            const uint16_t b = El[kEdgeRight + j];
            const uint16_t bU = j > 0 ? El[kEdgeRight + j - 1] : kBg;
            if (b != kBg && !(aU == a && bU == b)) union_global(s.P, base + a, lbase + b, cap, err);
            if (kConn8) {
                if (j > 0 && bU != kBg && aU != a) union_global(s.P, base + a, lbase + bU, cap, err);
                if (j + 1 < kTileH) {
                    const uint16_t bD = El[kEdgeRight + j + 1];
                    if (bD != kBg && aD != a) union_global(s.P, base + a, lbase + bD, cap, err);
                }
            }
        }
    }
    report(err);
}

// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) k_flatten(Scratch s, int cap) {
    const int t = blockIdx.x;
    const int n = s.nslots[t];
    int err = 0;
    for (int k = threadIdx.x; k < n; k += kThreads) {
        const uint32_t slot = (uint32_t)t * kSlots + (uint32_t)k;
        uint32_t key;
        const uint32_t root = find_global(s.P, slot, key, cap, err);
        if (root != slot && !err) ((volatile uint64_t *)s.P)[slot] = pack_slot(key, root);
    }
    report(err);
}

// ---------------------------------------------------------------------------
struct RelabelSmem {
    TileSmem tile;
    int slot_label[kSlots];
    int4 stage[kTileH * kTileW / 4];   // output tile, 16-byte chunks swizzled by row
};

__device__ __forceinline__ int stage_chunk(int row, int q) { return row * (kTileW / 4) + (q ^ (row & 7)); }

template <bool kConn8>
__global__ void __launch_bounds__(kThreads) k_relabel(ImageArgs a, Scratch s, int cap) {
    __shared__ RelabelSmem smr;
    TileSmem &sm = smr.tile;
    const int t = blockIdx.x;
    const int tx = t % a.ntx, ty = t / a.ntx;
    const int x0 = tx * kTileW, y0 = ty * kTileH;
    clear_tile_state(sm);

    uint32_t m, S;
    label_tile<kConn8>(sm, a.img, a.H, a.W, a.pitch, a.vec_ok, x0, y0, cap, m, S);
    number_border_roots(sm);

    // final label of each border component
    for (int k = threadIdx.x; k < sm.nslots; k += kThreads) {
        const uint64_t v = s.P[(size_t)t * kSlots + k];
        smr.slot_label[k] = (int)(uint32_t)(v >> 32) + 1;
    }
    __syncthreads();

    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int r = lane;
    const int rowbase = r * kTileW + kSubW * w;
    // every run start: root -> final label (in place; each lane touches only
    // the entries of its own row)
    for (uint32_t u = S; u; u &= u - 1) {
        const int n = rowbase + __ffs(u) - 1;
        const int root = sm.parent[swz(n)];
        const int lab = is_border_root(sm, root) ? smr.slot_label[border_slot(sm, root)]
                                                  : (int)node_key(root, x0, y0, a.W) + 1;
        sm.parent[swz(n)] = lab;
    }
    // expand run labels over the row into the staging tile
    {
        int cur = 0;
#pragma unroll
        for (int k = 0; k < kSubW / 4; ++k) {
            int v[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int c = 4 * k + j;
                if ((S >> c) & 1u) cur = sm.parent[swz(rowbase + c)];
                v[j] = ((m >> c) & 1u) ? cur : 0;
            }
            smr.stage[stage_chunk(r, (kSubW / 4) * w + k)] = make_int4(v[0], v[1], v[2], v[3]);
        }
    }
    __syncthreads();

    // coalesced write-out: a warp stores one 512-byte tile row per step
    for (int row = w; row < kTileH; row += kWarps) {
        const int y = y0 + row;
        if (y >= a.H) break;
        const int4 v = smr.stage[stage_chunk(row, lane)];
        const int x = x0 + 4 * lane;
        int32_t *dst = a.labels + (size_t)y * a.W + x;
        if (a.out_vec_ok && x + 4 <= a.W) {
            __stcs(reinterpret_cast<int4 *>(dst), v);
        } else {
            if (x + 0 < a.W) __stcs(dst + 0, v.x);
            if (x + 1 < a.W) __stcs(dst + 1, v.y);
            if (x + 2 < a.W) __stcs(dst + 2, v.z);
            if (x + 3 < a.W) __stcs(dst + 3, v.w);
        }
    }
    if (threadIdx.x == 0) report(sm.err);
}

}  // namespace ccl

// ---------------------------------------------------------------------------
// Host side of this translation unit.

namespace ccl {

size_t workspace_bytes(int H, int W) {
    const size_t ntx = ((size_t)W + kTileW - 1) / kTileW;
    const size_t nty = ((size_t)H + kTileH - 1) / kTileH;
    const size_t nt = ntx * nty;
    auto up = [](size_t v) { return (v + 255) & ~(size_t)255; };
    return up(nt * kEdge * sizeof(uint16_t)) + up(nt * kSlots * sizeof(uint64_t)) +
           up(nt * sizeof(int32_t));
}

static Scratch carve(void *ws, int H, int W) {
    const size_t ntx = ((size_t)W + kTileW - 1) / kTileW;
    const size_t nty = ((size_t)H + kTileH - 1) / kTileH;
    const size_t nt = ntx * nty;
    auto up = [](size_t v) { return (v + 255) & ~(size_t)255; };
    char *p = static_cast<char *>(ws);
    Scratch s;
    s.edges = reinterpret_cast<uint16_t *>(p);
    p += up(nt * kEdge * sizeof(uint16_t));
    s.P = reinterpret_cast<uint64_t *>(p);
    p += up(nt * kSlots * sizeof(uint64_t));
    s.nslots = reinterpret_cast<int32_t *>(p);
    return s;
}

// ---------------------------------------------------------------------------
// Per-kernel timing for benchmarks: when on, an event is recorded on the
// launching stream before the first kernel of a call and after each kernel;
// consecutive events bracket one kernel.  Completed events are folded into
// per-kind sums and returned to a pool, so long runs hold few events.

namespace {

struct TimingRec {
    int kind;
    cudaEvent_t a, b;
};

struct TimingState {
    std::mutex mu;
    bool on = false;
    std::vector<cudaEvent_t> pool;
    std::deque<TimingRec> pending;
    double ms[kKernelKinds] = {};
    long long count[kKernelKinds] = {};
} g_timing;

cudaEvent_t timing_event() {
    if (!g_timing.pool.empty()) {
        cudaEvent_t e = g_timing.pool.back();
        g_timing.pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

void timing_fold(bool wait) {
    while (!g_timing.pending.empty()) {
        TimingRec r = g_timing.pending.front();
        if (wait) {
            cudaEventSynchronize(r.b);
        } else if (cudaEventQuery(r.b) != cudaSuccess) {
            cudaGetLastError();
            break;
        }
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
            g_timing.ms[r.kind] += ms;
            g_timing.count[r.kind] += 1;
        } else {
            cudaGetLastError();
        }
        g_timing.pending.pop_front();
        // r.b opens the next record of the same call, so only r.a is free
        // now; the last record of a call frees its closing event as well.
        g_timing.pool.push_back(r.a);
        if (r.kind == kKernelKinds - 1) g_timing.pool.push_back(r.b);
    }
}

// Records an event on `s` and, when `kind` >= 0, closes a record for the
// kernel launched since `prev`.  Returns the new event (nullptr when off).
cudaEvent_t timing_mark(cudaStream_t s, cudaEvent_t prev, int kind) {
    std::lock_guard<std::mutex> lk(g_timing.mu);
    if (!g_timing.on) return nullptr;
    timing_fold(false);
    cudaEvent_t e = timing_event();
    cudaEventRecord(e, s);
    if (kind >= 0 && prev) g_timing.pending.push_back({kind, prev, e});
    return e;
}

}  // namespace

void timing_enable(bool on) {
    std::lock_guard<std::mutex> lk(g_timing.mu);
    timing_fold(true);
    g_timing.on = on;
    for (int k = 0; k < kKernelKinds; ++k) {
        g_timing.ms[k] = 0.0;
        g_timing.count[k] = 0;
    }
}

int timing_read(double *ms, long long *count, int n) {
    std::lock_guard<std::mutex> lk(g_timing.mu);
    timing_fold(true);
    for (int k = 0; k < n && k < kKernelKinds; ++k) {
        ms[k] = g_timing.ms[k];
        count[k] = g_timing.count[k];
    }
    return kKernelKinds;
}

const char *kernel_kind_name(int k) {
    static const char *names[kKernelKinds] = {"k_local_border", "k_block_merge", "k_flatten", "k_relabel"};
    return (k >= 0 && k < kKernelKinds) ? names[k] : "";
}

int launch_label(const uint8_t *img, int H, int W, size_t pitch, int conn, int32_t *labels, void *ws,
                 cudaStream_t stream, int cap) {
    ImageArgs a;
    a.img = img;
    a.labels = labels;
    a.pitch = pitch;
    a.H = H;
    a.W = W;
    a.ntx = (W + kTileW - 1) / kTileW;
    a.nty = (H + kTileH - 1) / kTileH;
    a.vec_ok = ((reinterpret_cast<uintptr_t>(img) | pitch) & 15) == 0;
    a.out_vec_ok = (reinterpret_cast<uintptr_t>(labels) & 15) == 0 && (W & 3) == 0;
    const Scratch s = carve(ws, H, W);
    const unsigned nt = (unsigned)a.ntx * (unsigned)a.nty;
    // Default caps: a find walks a strictly decreasing chain, so it cannot
    // take more steps than there are nodes (slots); no valid input reaches them.
    const long long slots = (long long)nt * kSlots + 16;
    const int local_cap = cap > 0 ? cap : 2 * kNodes;
    const int global_cap = cap > 0 ? cap : (int)(slots < (1LL << 30) ? slots : (1LL << 30));
    cudaEvent_t ev = timing_mark(stream, nullptr, -1);
    if (conn == 8) {
        k_local_border<true><<<nt, kThreads, 0, stream>>>(a, s, local_cap);
        ev = timing_mark(stream, ev, kKindLocal);
        k_block_merge<true><<<nt, kThreads, 0, stream>>>(s, a.ntx, a.nty, global_cap);
        ev = timing_mark(stream, ev, kKindMerge);
        k_flatten<<<nt, kThreads, 0, stream>>>(s, global_cap);
        ev = timing_mark(stream, ev, kKindFlatten);
        k_relabel<true><<<nt, kThreads, 0, stream>>>(a, s, local_cap);
        ev = timing_mark(stream, ev, kKindRelabel);
    } else {
        k_local_border<false><<<nt, kThreads, 0, stream>>>(a, s, local_cap);
        ev = timing_mark(stream, ev, kKindLocal);
        k_block_merge<false><<<nt, kThreads, 0, stream>>>(s, a.ntx, a.nty, global_cap);
        ev = timing_mark(stream, ev, kKindMerge);
        k_flatten<<<nt, kThreads, 0, stream>>>(s, global_cap);
        ev = timing_mark(stream, ev, kKindFlatten);
        k_relabel<false><<<nt, kThreads, 0, stream>>>(a, s, local_cap);
        ev = timing_mark(stream, ev, kKindRelabel);
    }
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int read_and_clear_device_error(int *value) {
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_device_error, sizeof(int)) != cudaSuccess) return -1;
    if (v) {
        const int zero = 0;
        if (cudaMemcpyToSymbol(g_device_error, &zero, sizeof(int)) != cudaSuccess) return -1;
    }
    *value = v;
    return 0;
}

}  // namespace ccl
