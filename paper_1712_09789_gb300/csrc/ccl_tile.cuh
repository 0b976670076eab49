// ccl_tile.cuh -- device building blocks of the block-based labeller.
//
// Tile geometry.  A CTA owns a kTileH x kTileW tile of the image (32 x 128).
// Each of its 4 warps owns a 32-column strip; lane r of a warp holds row r of
// its strip as one 32-bit mask (bit c = pixel (r, 32*w + c)).  Everything the
// paper does per pixel in Kernel 1 is done here per row mask with bit
// operations, and the label-equivalence lists are kept only at run starts.
//
// Node ids.  Inside a tile, pixel (r, x) has node id n = r*kTileW + x.  Node
// order equals raster order restricted to the tile, so the minimum node of a
// tile-local component is also its minimum global raster position (the ID
// conversion of Sec. 3.1.4 preserves order).  Shared-memory slot of node n is
// swz(n): the low five bits are XORed with the row so that lanes holding
// different rows of the same column hit different banks.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace ccl {

constexpr int kSubW = 32;                    // columns per warp strip
constexpr int kTileH = 32;                   // rows per tile (one per lane)
constexpr int kWarps = 4;                    // strips per tile
constexpr int kTileW = kSubW * kWarps;       // 128
constexpr int kTileWLog2 = 7;
constexpr int kNodes = kTileH * kTileW;      // 4096
constexpr int kThreads = 32 * kWarps;        // 128
// A component that touches the tile border meets the border cycle of
// 2*(kTileW + kTileH) - 4 pixels in at least one maximal foreground arc, and
// the cycle holds at most half its length in arcs.
constexpr int kSlots = kTileW + kTileH;      // >= (2*(W+H)-4)/2 border components
// Border record per tile: top row, bottom row, left column, right column.
constexpr int kEdgeTop = 0;
constexpr int kEdgeBottom = kTileW;
constexpr int kEdgeLeft = 2 * kTileW;
constexpr int kEdgeRight = 2 * kTileW + kTileH;
constexpr int kEdge = 2 * kTileW + 2 * kTileH;
constexpr uint16_t kBg = 0xFFFF;
constexpr unsigned kFull = 0xFFFFFFFFu;

// device error word bits
constexpr int kErrLocalCap = 1;
constexpr int kErrGlobalCap = 2;

__device__ __forceinline__ int swz(int n) { return n ^ ((n >> kTileWLog2) & 31); }

// bits 0..c set (c in [0,31]); c == 31 wraps to all ones
__device__ __forceinline__ uint32_t upto(int c) { return (2u << c) - 1u; }

// highest set bit index (v != 0)
__device__ __forceinline__ int hibit(uint32_t v) { return 31 - __clz(v); }

// 4 bytes -> 4 bits, bit k set iff byte k is nonzero.  The add sets bit 7 of
// a byte when its low seven bits are nonzero (no carry leaves the byte); the
// multiply gathers the four bit-7s into bits 28..31 without overlapping
// partial products.
__device__ __forceinline__ uint32_t nz4(uint32_t w) {
    uint32_t t = (((w & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | w) & 0x80808080u;
    return (t * 0x00204081u) >> 28;
}

__device__ __forceinline__ uint32_t nz16(uint4 v) {
    return nz4(v.x) | (nz4(v.y) << 4) | (nz4(v.z) << 8) | (nz4(v.w) << 12);
}

__device__ __forceinline__ uint4 ldg_stream16(const uint8_t *p) {
    uint4 v;
    asm volatile("ld.global.nc.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
}

// Row mask of the 32 pixels (y, x .. x+31).  Pixels outside the image are
// background.  `vec_ok` says that img and pitch are 16-byte aligned.
__device__ __forceinline__ uint32_t load_row_mask(const uint8_t *img, size_t pitch, int H, int W,
                                                  int y, int x, bool vec_ok) {
    if (y >= H || x >= W) return 0u;
    const uint8_t *p = img + (size_t)y * pitch + x;
    if (vec_ok && x + 32 <= W) {
        uint4 a = ldg_stream16(p);
        uint4 b = ldg_stream16(p + 16);
        return nz16(a) | (nz16(b) << 16);
    }
    int n = W - x < 32 ? W - x : 32;
    uint32_t m = 0;
    for (int i = 0; i < n; ++i) m |= (uint32_t)(__ldg(p + i) != 0) << i;
    return m;
}

// ---------------------------------------------------------------------------
// Shared-memory union-find over node ids.  parent[swz(n)] <= n always; a root
// has parent == itself.  Links go from the larger root to the smaller, so a
// root is the minimum node of its set (Sec. 3.1.3: "make the larger one point
// to the smaller one", done atomically because several lanes may update the
// same list at once).

__device__ __forceinline__ int find_smem(volatile int *parent, int x, int cap, int &err) {
    for (int i = 0; i < cap; ++i) {
        int p = parent[swz(x)];
        if (p == x) return x;
        x = p;
    }
    err |= kErrLocalCap;
    return x;
}

// Union of the sets of a and b.  atomicMin keeps parent links monotone; when
// the min lands on a node that had meanwhile been linked elsewhere, the old
// parent is merged with b in the next round, so no equivalence is lost.
__device__ __forceinline__ void union_smem(int *parent, int a, int b, int cap, int &err) {
    volatile int *vp = parent;
    for (int i = 0; i < cap; ++i) {
        a = find_smem(vp, a, cap, err);
        b = find_smem(vp, b, cap, err);
        if (a == b) return;
        if (a < b) { int t = a; a = b; b = t; }
        int old = atomicMin(parent + swz(a), b);
        if (old == a) return;
        a = old;
    }
    err |= kErrLocalCap;
}

// ---------------------------------------------------------------------------
// Global union-find over border slots.  Slot s = tile * kSlots + k stands for
// the k-th border-touching component of a tile.  P[s] packs
// (key of parent << 32) | parent slot, where a slot's key is the minimum
// global raster position of its component; a root has P[s] == (key(s)<<32)|s.
// atomicMin on the packed word links the root with the larger key under the
// root with the smaller key (Kernel 2: "larger label pointing to the smaller").

__device__ __forceinline__ uint64_t pack_slot(uint32_t key, uint32_t slot) {
    return ((uint64_t)key << 32) | slot;
}

__device__ __forceinline__ uint32_t find_global(const uint64_t *P, uint32_t s, uint32_t &key, int cap,
                                                int &err) {
    const volatile uint64_t *vp = P;
    for (int i = 0; i < cap; ++i) {
        uint64_t v = vp[s];
        uint32_t p = (uint32_t)v;
        if (p == s) { key = (uint32_t)(v >> 32); return s; }
        s = p;
    }
    err |= kErrGlobalCap;
    key = 0xFFFFFFFFu;
    return s;
}

__device__ __forceinline__ void union_global(uint64_t *P, uint32_t a, uint32_t b, int cap, int &err) {
    for (int i = 0; i < cap; ++i) {
        uint32_t ka, kb;
        a = find_global(P, a, ka, cap, err);
        b = find_global(P, b, kb, cap, err);
        if (a == b || err) return;
        if (ka < kb) { uint32_t t = a; a = b; b = t; t = ka; ka = kb; kb = t; }
        unsigned long long old = atomicMin((unsigned long long *)(P + a),
                                           (unsigned long long)pack_slot(kb, b));
        if (old == pack_slot(ka, a)) return;
        a = (uint32_t)old;
    }
    err |= kErrGlobalCap;
}

// Column of the row above that a contact marked at bit c touches: c itself
// for an overlap, c - 1 for an up-left and c + 1 for an up-right diagonal
// (the up-left reading wins when a bit carries both).
__device__ __forceinline__ int upper_column(int c, uint32_t DR, uint32_t DL) {
    const int dl = (int)((DL >> c) & 1u);
    const int dr = (int)((DR >> c) & 1u) & (dl ^ 1);
    return c + dr - dl;
}

// ---------------------------------------------------------------------------
// Per-tile shared state.

struct TileSmem {
    int parent[kNodes];                 // union-find, indexed by swz(node)
    uint32_t rowm[kWarps][kTileH];      // foreground masks per strip row
    uint32_t runs[kWarps][kTileH];      // run-start masks per strip row
    uint32_t border[kNodes / 32];       // roots touching the tile border
    uint32_t prefix[kNodes / 32];       // exclusive popcount prefix of border[]
    int nslots;
    int err;
};

// Local labelling of one tile (Kernel 1 up to the ID conversion).  On return
// (after a __syncthreads) parent[swz(n)] holds, for every run start n, the
// minimum node of n's tile-local component; this lane's row mask and run
// starts are returned in m and S.
//
// Phases (Sec. 3.1):
//   initialization  row masks staged from global memory;
//   coarse labeling row connection -- each maximal run of a row is one list
//                   whose root is the run start (bit ops, no iteration);
//                   column connection -- a run with foreground above links
//                   to the first run above that it touches; the lists are
//                   then unified top-down so that every run start points at
//                   the root of its coarse list;
//   refinement      the remaining contacts between a run and further runs
//                   above, and the contacts across the strips of the tile,
//                   are merged with atomic unions; a final root-find
//                   compresses every run start onto its root.
template <bool kConn8>
__device__ __forceinline__ void label_tile(TileSmem &sm, const uint8_t *img, int H, int W, size_t pitch,
                                           bool vec_ok, int x0, int y0, int cap, uint32_t &m_out,
                                           uint32_t &S_out) {
    const int lane = threadIdx.x & 31;
    const int w = threadIdx.x >> 5;
    const int r = lane;
    int err = 0;

    // -- initialization: this lane's row of the strip as a bit mask
    const uint32_t m = load_row_mask(img, pitch, H, W, y0 + r, x0 + kSubW * w, vec_ok);
    uint32_t mu = __shfl_up_sync(kFull, m, 1);
    if (lane == 0) mu = 0;
    const uint32_t S = m & ~(m << 1);              // run starts
    uint32_t Su = __shfl_up_sync(kFull, S, 1);
    if (lane == 0) Su = 0;
    sm.rowm[w][r] = m;
    sm.runs[w][r] = S;

    // -- coarse labeling, column connection.  A contact between a run A of
    // this row and a run B of the row above is marked once, at one pixel of A:
    // the first column of their overlap, or (8-connectivity) the end pixel of
    // A that touches B only diagonally.
    const uint32_t ov = m & mu;
    uint32_t T = ov & ~(ov << 1);
    uint32_t DR = 0, DL = 0;
    if (kConn8) {
        DR = m & ~(m >> 1) & (mu >> 1) & ~mu;      // up-right contact at A's last pixel
        DL = S & (mu << 1) & ~mu;                  // up-left contact at A's first pixel
        T |= DR | DL;
    }
    // Per run, keep the lowest contact: F covers each run from its first
    // contact to its end (the add clears exactly that span), so a contact
    // with F set just left of it is not the first of its run.
    const uint32_t F = m & ~((m + T) & ~T);
    const uint32_t FS = T & ~(F << 1);
    const uint32_t X = T ^ FS;                     // later contacts: refinement
    // A one-pixel run can touch the row above at both diagonals, which marks
    // the same bit twice; the bit then stands for the up-left contact and the
    // up-right contact is merged in the refinement.
    const uint32_t XR = DR & DL;

    const int rowbase = r * kTileW + kSubW * w;
    uint32_t HS = 0;                               // run starts with a coarse link
    for (uint32_t t = FS; t; t &= t - 1) {
        const int c = __ffs(t) - 1;
        const int a0 = hibit(S & upto(c));
        const int b0 = hibit(Su & upto(upper_column(c, DR, DL)));
        sm.parent[swz(rowbase + a0)] = rowbase - kTileW + b0;
        HS |= 1u << a0;
    }
    for (uint32_t t = S & ~HS; t; t &= t - 1) {
        const int a0 = __ffs(t) - 1;
        sm.parent[swz(rowbase + a0)] = rowbase + a0;
    }
    __syncwarp();

    // -- unification of the coarse lists, top-down with lane = column: the
    // parent of a linked run start lies in the row above, whose entries are
    // already roots, so one hop makes it a root as well.
    {
        const int c = lane;
        uint32_t rows_with_links = __ballot_sync(kFull, HS != 0) & ~1u;
        for (; rows_with_links; rows_with_links &= rows_with_links - 1) {
            const int rr = __ffs(rows_with_links) - 1;
            const uint32_t hs = __shfl_sync(kFull, HS, rr);
            if ((hs >> c) & 1u) {
                const int n = rr * kTileW + kSubW * w + c;
                const int p = sm.parent[swz(n)];
                sm.parent[swz(n)] = sm.parent[swz(p)];
            }
            __syncwarp();
        }
    }
    __syncthreads();

    // -- refinement: further contacts with the row above ...
    for (uint32_t t = X; t; t &= t - 1) {
        const int c = __ffs(t) - 1;
        const int a0 = hibit(S & upto(c));
        const int b0 = hibit(Su & upto(upper_column(c, DR, DL)));
        union_smem(sm.parent, rowbase + a0, rowbase - kTileW + b0, cap, err);
    }
    for (uint32_t t = XR; t; t &= t - 1) {
        const int c = __ffs(t) - 1;               // a one-pixel run: c is its start
        union_smem(sm.parent, rowbase + c, rowbase - kTileW + hibit(Su & upto(c + 1)), cap, err);
    }
    // ... and contacts across the seam with the strip on the left.
    if (w > 0 && (m & 1u)) {
        const int me = rowbase;
        const int lb = r * kTileW + kSubW * (w - 1);
        const uint32_t mL = sm.rowm[w - 1][r];
        if (mL >> 31) union_smem(sm.parent, me, lb + hibit(sm.runs[w - 1][r]), cap, err);
        if (kConn8) {
            if (r > 0 && (sm.rowm[w - 1][r - 1] >> 31))
                union_smem(sm.parent, me, lb - kTileW + hibit(sm.runs[w - 1][r - 1]), cap, err);
            if (r + 1 < kTileH && (sm.rowm[w - 1][r + 1] >> 31))
                union_smem(sm.parent, me, lb + kTileW + hibit(sm.runs[w - 1][r + 1]), cap, err);
        }
    }
    __syncthreads();

    // -- final root-find for every run start (no unions run any more, so a
    // concurrent write seen here is always an ancestor of the node read)
    {
        volatile int *vp = sm.parent;
        for (uint32_t t = S; t; t &= t - 1) {
            const int n = rowbase + __ffs(t) - 1;
            vp[swz(n)] = find_smem(vp, n, cap, err);
        }
    }
    if (err) atomicOr(&sm.err, err);
    __syncthreads();
    m_out = m;
    S_out = S;
}

// Mark every root that owns a border pixel of the tile and number those roots
// by increasing node id (exclusive prefix of popcounts).  Needs sm.border
// cleared beforehand; ends with a __syncthreads.
__device__ __forceinline__ void number_border_roots(TileSmem &sm) {
    const int lane = threadIdx.x & 31;
    const int w = threadIdx.x >> 5;
    // top and bottom rows, lane = column
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int rr = k ? kTileH - 1 : 0;
        const uint32_t m = sm.rowm[w][rr];
        if ((m >> lane) & 1u) {
            const int a0 = hibit(sm.runs[w][rr] & upto(lane));
            const int root = sm.parent[swz(rr * kTileW + kSubW * w + a0)];
            atomicOr(&sm.border[root >> 5], 1u << (root & 31));
        }
    }
    // left column (strip 0) and right column (last strip), lane = row
    if (w == 0 && (sm.rowm[0][lane] & 1u)) {
        const int root = sm.parent[swz(lane * kTileW)];
        atomicOr(&sm.border[root >> 5], 1u << (root & 31));
    }
    if (w == kWarps - 1 && (sm.rowm[w][lane] >> 31)) {
        const int root = sm.parent[swz(lane * kTileW + kSubW * w + hibit(sm.runs[w][lane]))];
        atomicOr(&sm.border[root >> 5], 1u << (root & 31));
    }
    __syncthreads();
    if (w == 0) {
        // 128 words, 4 per lane
        uint32_t c[4];
        uint32_t s = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) { c[k] = __popc(sm.border[lane * 4 + k]); s += c[k]; }
        uint32_t incl = s;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t v = __shfl_up_sync(kFull, incl, d);
            if (lane >= d) incl += v;
        }
        uint32_t run = incl - s;
#pragma unroll
        for (int k = 0; k < 4; ++k) { sm.prefix[lane * 4 + k] = run; run += c[k]; }
        if (lane == 31) sm.nslots = (int)incl;
    }
    __syncthreads();
}

__device__ __forceinline__ int border_slot(const TileSmem &sm, int root) {
    const uint32_t word = sm.border[root >> 5];
    return (int)(sm.prefix[root >> 5] + __popc(word & ((1u << (root & 31)) - 1u)));
}

__device__ __forceinline__ bool is_border_root(const TileSmem &sm, int root) {
    return (sm.border[root >> 5] >> (root & 31)) & 1u;
}

// ID conversion (Sec. 3.1.4): node -> global raster position.
__device__ __forceinline__ uint32_t node_key(int node, int x0, int y0, int W) {
    return (uint32_t)(y0 + (node >> kTileWLog2)) * (uint32_t)W + (uint32_t)(x0 + (node & (kTileW - 1)));
}

}  // namespace ccl
