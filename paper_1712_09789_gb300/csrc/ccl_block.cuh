// ccl_block.cuh -- device building blocks of the block-based labeller.
//
// Geometry.  A CTA owns a block of (32 * BLX) x (kLH * BLY) pixels and has one
// thread per lane tile of 32 columns x kLH rows (tx = t % BLX, ty = t / BLX).
// Short lane tiles keep each thread's chain of dependent steps short, so a
// mid-size image still puts enough warps on every SM.
// A thread holds each row of its lane tile as a 32-bit mask (bit c = column
// c).  The block shape (BLX, BLY) is a template parameter so that the batched
// path can pick it per workload.
//
// Bands and pieces.  A lane tile is cut into bands of two rows.  A piece is
// one connected component of a band, and it is found by bit operations: the
// two pixels of a column of a band always touch, so a component is a run of
// columns, each linked to the next (see band_link).  Under 8-connectivity
// every pixel of a column is adjacent to every pixel of the next (|dx| <= 1,
// |dy| <= 1), so the pieces are the runs of the OR of the two rows; under
// 4-connectivity a run of the OR splits where its columns meet only
// diagonally.  There are fewer pieces than row runs, so the label-equivalence
// work shrinks.  Pieces are numbered per lane tile in band order, then column
// order, which is recomputable from the masks by a popcount.
//
// Label-equivalence lists.  Piece `loc` of thread t has the id
// (t << kLocBits) | loc
// and one 16-bit entry in shared memory: a root holds kRoot | key, key being
// the block raster position (row * block width + column) of the smallest
// pixel of its list; any other entry holds the id of its parent.  Links go
// from the larger key to the smaller (Sec. 3.1.3 and 3.2), so the root of a
// component carries the component's smallest block raster position.  Entry of
// id i lives at par[(i & (capacity - 1)) * threads + (i >> kLocBits)], so 32
// lanes touching
// their own piece loc hit 32 consecutive half-words.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace ccl {

constexpr int kLW = 32;                 // lane tile width (bits of a row mask)
constexpr uint16_t kRoot = 0x8000;
constexpr uint16_t kBorderRoot = 0x4000;  // entry of a root once its border slot is known: kBorderRoot | slot
constexpr uint16_t kBg = 0xFFFF;
constexpr uint16_t kBorderFlag = 0x8000;  // per-piece value: border slot, else block key
constexpr unsigned kFull = 0xFFFFFFFFu;

constexpr int kErrLocalCap = 1;
constexpr int kErrGlobalCap = 2;

constexpr int ilog2(int v) { return v <= 1 ? 0 : 1 + ilog2(v / 2); }

template <int BLX_, int BLY_, int LH_>
struct Geo {
    static constexpr int BLX = BLX_;                  // lane tiles across a block
    static constexpr int BLY = BLY_;                  // lane tiles down a block
    static constexpr int kLH = LH_;                   // lane tile height (rows of a thread)
    static constexpr int kThreads = BLX * BLY;
    static constexpr int kPieceCap = kLH * 16;        // elements per lane tile: at most 32 per two-row band
    static constexpr int kLocBits = ilog2(kPieceCap); // piece index bits of a piece id
    static constexpr int kVChunks = kPieceCap / 8;    // 8 two-byte values per 16-byte chunk
    static constexpr int kBW = kLW * BLX;
    static constexpr int kBH = kLH * BLY;
    static constexpr int kBWLog2 = ilog2(kBW);
    static constexpr int kBLXLog2 = ilog2(BLX);
    // A component touching the block border meets the border cycle
    // (2*(kBW + kBH) - 4 pixels) in at least one maximal foreground arc, and
    // the cycle holds at most half its length in arcs.
    static constexpr int kSlots = kBW + kBH;
    static constexpr int kEdgeTop = 0;
    static constexpr int kEdgeBottom = kBW;
    static constexpr int kEdgeLeft = 2 * kBW;
    static constexpr int kEdgeRight = 2 * kBW + kBH;
    static constexpr int kEdge = 2 * kBW + 2 * kBH;
    // ids carry the thread index above kLocBits piece bits and stay below
    // kBorderRoot (an entry below it is a parent id); block keys fit 15 bits
    static_assert(kThreads >= 32 && (kThreads << kLocBits) <= kBorderRoot && (kThreads & (kThreads - 1)) == 0,
                  "32..256 threads, a power of two");
    static_assert((BLX & (BLX - 1)) == 0, "BLX must be a power of two");
    static_assert(kLH % 4 == 0 && (kPieceCap & (kPieceCap - 1)) == 0, "lane tiles of 4 or 8 rows");
    static_assert(kBW * kBH <= 32768, "block keys must fit 15 bits");
    static_assert((kEdge * 2) % 16 == 0, "border records must stay 16-byte aligned");
};

// Band layout of a lane tile for one connectivity: bands of two rows; a band
// holds at most 16 pieces under 8-connectivity (pieces are runs of the OR of
// its rows), 32 under 4-connectivity (one per column at most).
template <bool kConn8, int kLH>
struct Bands {
    static constexpr int kRows = 2;                // rows per band
    static constexpr int kN = kLH / kRows;         // bands per lane tile
    static constexpr int kCap = (kConn8 ? 16 : 32) * kN;  // pieces per lane tile
    static constexpr int kVChunks = kCap / 8;
};

// bits 0..c set (c in [0,31]); c == 31 wraps to all ones
__device__ __forceinline__ uint32_t upto(int c) { return (2u << c) - 1u; }
__device__ __forceinline__ int hibit(uint32_t v) { return 31 - __clz(v); }
__device__ __forceinline__ int lobit(uint32_t v) { return __ffs(v) - 1; }

// 4 bytes -> 4 bits, bit k set iff byte k is nonzero.  The add sets bit 7 of
// a byte when its low seven bits are nonzero (no carry leaves the byte); the
// multiply gathers the four bit-7s into bits 28..31 without overlapping
// partial products.
__device__ __forceinline__ uint32_t nz4(uint32_t w) {
    const uint32_t t = (((w & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | w) & 0x80808080u;
    return (t * 0x00204081u) >> 28;
}

__device__ __forceinline__ uint32_t nz16(uint4 v) {
    return nz4(v.x) | (nz4(v.y) << 4) | (nz4(v.z) << 8) | (nz4(v.w) << 12);
}

__device__ __forceinline__ uint4 ldg_nc16(const void *p) {
    uint4 v;
    asm volatile("ld.global.nc.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
}

// Programmatic dependent launch (griddepcontrol): a kernel launched with
// programmatic stream serialisation may start while the kernel before it on
// the stream still runs.  grid_dependency_wait() blocks until that kernel has
// completed and its memory is visible (a no-op for a kernel launched without
// the attribute); grid_launch_dependents() lets the next such kernel start
// once every CTA of this grid has called it or exited.
__device__ __forceinline__ void grid_dependency_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;"); }

// Run mask of bits a0..a1.  a1 == 31 wraps 2u << 31 to 0, which still gives
// the bits a0..31.
__device__ __forceinline__ uint32_t run_bits(int a0, int a1) { return (2u << a1) - (1u << a0); }

// Columns of the neighbouring row that touch the given pixels of a row: the
// pixels themselves, widened by one column on each side for 8-connectivity.
template <bool kConn8>
__device__ __forceinline__ uint32_t touch_range(uint32_t rm) {
    return kConn8 ? (rm | (rm << 1) | (rm >> 1)) : rm;
}

// Links of a band with rows A (upper) and B (lower): bit c is set when
// columns c and c+1 hold pixels of one piece.  The pixels of one column of a
// band always touch.  Under 8-connectivity any pixel of a column touches any
// pixel of the next one, so two occupied columns are linked; under
// 4-connectivity only a row holding both pixels links them.
template <bool kConn8>
__device__ __forceinline__ uint32_t band_link(uint32_t A, uint32_t B) {
    const uint32_t OR = A | B;
    return kConn8 ? (OR & (OR >> 1)) : ((A & (A >> 1)) | (B & (B >> 1)));
}

// First and last columns of the band's pieces.
template <bool kConn8>
__device__ __forceinline__ uint32_t band_starts(uint32_t A, uint32_t B) {
    return (A | B) & ~(band_link<kConn8>(A, B) << 1);
}
template <bool kConn8>
__device__ __forceinline__ uint32_t band_ends(uint32_t A, uint32_t B) {
    return (A | B) & ~band_link<kConn8>(A, B);
}

// Coarse-labelling variants of Sec. 4.2: C2FL (0, the method), RC2FL (1,
// coarse labelling along rows only), CC2FL (2, along columns only), NC2FL (3,
// neither; the refinement does all the merging).  Along rows: the elements of
// a band are its pieces (else every occupied column of a band is an element
// of its own, and the links between neighbouring columns are refined).  Along
// columns: an element takes the first element above it that it touches as
// parent (else every contact with the band above is refined).
template <bool kConn8, int kMode, int kLH>
struct Variant {
    static constexpr bool kRow = kMode == 0 || kMode == 1;
    static constexpr bool kCol = kMode == 0 || kMode == 2;
    static constexpr int kCap = ((kConn8 && kRow) ? 16 : 32) * (kLH / 2);  // elements per lane tile
};

template <bool kConn8, bool kRow>
__device__ __forceinline__ uint32_t elem_starts(uint32_t A, uint32_t B) {
    return kRow ? band_starts<kConn8>(A, B) : (A | B);
}
template <bool kConn8, bool kRow>
__device__ __forceinline__ uint32_t elem_ends(uint32_t A, uint32_t B) {
    return kRow ? band_ends<kConn8>(A, B) : (A | B);
}

// Last column of the piece (run of `ends`' mask) holding column u.
__device__ __forceinline__ int piece_end(uint32_t ends, int u) { return u + lobit(ends >> u); }

// ---------------------------------------------------------------------------
// Shared-memory label-equivalence lists of one block.

// Id of piece `loc` of the lane tile of thread t.
template <class G>
__device__ __forceinline__ int piece_id(int t, int loc) { return (t << G::kLocBits) | loc; }

// (masked on both fields, so no entry value can address outside the table)
template <class G, int kCap>
__device__ __forceinline__ int par_index(int id) {
    return (id & (kCap - 1)) * G::kThreads + ((id >> G::kLocBits) & (G::kThreads - 1));
}

// Root of id and the root's entry.  Path halving rewrites only non-root
// entries, and links are only ever made on roots (by CAS), so the two never
// overwrite each other.
template <class G, int kCap>
__device__ __forceinline__ int find_root(volatile uint16_t *par, int x, uint16_t &rentry, int cap, int &err,
                                         unsigned *ops = nullptr) {
    for (int i = 0; i < cap; ++i) {
        if (ops) ++ops[1];
        const uint16_t e = par[par_index<G, kCap>(x)];
        if (e & kRoot) { rentry = e; return x; }
        const uint16_t g = par[par_index<G, kCap>(e)];
        if (g & kRoot) { rentry = g; return e; }
        par[par_index<G, kCap>(x)] = g;
        x = g;
    }
    err |= kErrLocalCap;
    rentry = kRoot;
    return x;
}

// Root of id without writing anything: used once no list changes any more,
// by threads that then store the root into entries.  (A halving find there
// could store an older grandparent over an entry that another thread had
// already set to its root.)
template <class G, int kCap>
__device__ __forceinline__ int find_root_ro(const volatile uint16_t *par, int x, int cap, int &err) {
    for (int i = 0; i < cap; ++i) {
        const uint16_t e = par[par_index<G, kCap>(x)];
        if (e & kRoot) return x;
        x = e;
    }
    err |= kErrLocalCap;
    return x;
}

// Merge the lists of a and b when both belong to the calling thread's lane
// tile and no other thread reads or writes its entries yet: plain finds and
// a plain store, the root with the larger key hung under the other.
template <class G, int kCap>
__device__ __forceinline__ void union_private(uint16_t *par, int a, int b, int cap, int &err,
                                              unsigned *ops = nullptr) {
    uint16_t ea, eb;
    if (ops) ++ops[0];
    a = find_root<G, kCap>(par, a, ea, cap, err, ops);
    b = find_root<G, kCap>(par, b, eb, cap, err, ops);
    if (a == b) return;
    if ((ea & 0x7FFF) < (eb & 0x7FFF)) par[par_index<G, kCap>(b)] = (uint16_t)a;
    else par[par_index<G, kCap>(a)] = (uint16_t)b;
}

// Merge the lists of ids a and b, called by all 32 lanes of a warp together
// (lanes with valid == false only keep step): the root with the larger key is
// hung under the root with the smaller key.  A failed CAS means the root
// changed meanwhile; the round repeats until no lane needs another, so the
// warp stays converged between rounds.
template <class G, int kCap>
__device__ __forceinline__ void union_block_sync(uint16_t *par, bool valid, int a, int b, int cap, int &err,
                                                 unsigned *ops = nullptr) {
    volatile uint16_t *vp = par;
    bool pend = valid;
    if (ops && valid) ++ops[0];
    for (int i = 0; __any_sync(kFull, pend); ++i) {
        if (pend) {
            uint16_t ea, eb;
            a = find_root<G, kCap>(vp, a, ea, cap, err, ops);
            b = find_root<G, kCap>(vp, b, eb, cap, err, ops);
            if (a == b || err) {
                pend = false;
            } else {
                if ((ea & 0x7FFF) < (eb & 0x7FFF)) {
                    const int t = a; a = b; b = t;
                    const uint16_t u = ea; ea = eb; eb = u;
                }
                if (ops) ++ops[2];
                const unsigned short old = atomicCAS(reinterpret_cast<unsigned short *>(par + par_index<G, kCap>(a)),
                                                     (unsigned short)ea, (unsigned short)b);
                if (old == ea) pend = false;
            }
        }
        if (i >= cap) {
            if (pend) err |= kErrLocalCap;
            break;
        }
    }
}

// ---------------------------------------------------------------------------
// Global union-find over border slots.  Slot s = block * slots-per-block + k
// stands for the k-th border-touching component of a block; P[s] packs
// (key of parent << 32) | parent slot, the key being the component's minimum
// global raster position; a root has P[s] == (key(s) << 32) | s.  atomicMin on
// the packed word hangs the root with the larger key under the smaller one.
// Every walk checks pointers against `bound` (the number of slots).

__device__ __forceinline__ uint64_t pack_slot(uint32_t key, uint32_t slot) {
    return ((uint64_t)key << 32) | slot;
}

// Root of slot s and its key; halves the path on the way (plain stores of an
// ancestor, which a concurrent atomicMin link on a root cannot lose: the
// linking thread retries with whatever value it displaced).
__device__ __forceinline__ uint32_t find_global(uint64_t *P, uint32_t s, uint32_t &key, int cap, int &err,
                                                uint32_t bound) {
    volatile uint64_t *vp = P;
    for (int i = 0; i < cap; ++i) {
        const uint64_t v = vp[s];
        const uint32_t p = (uint32_t)v;
        if (p == s) { key = (uint32_t)(v >> 32); return s; }
        if (p >= bound) break;
        const uint64_t g = vp[p];
        if ((uint32_t)g >= bound) break;
        if ((uint32_t)g == p) { key = (uint32_t)(g >> 32); return p; }
        vp[s] = g;
        s = (uint32_t)g;
    }
    err |= kErrGlobalCap;
    key = 0xFFFFFFFFu;
    return s;
}

// Read-only root-find, for threads that only need the final key.
__device__ __forceinline__ uint32_t find_global_ro(const uint64_t *P, uint32_t s, uint32_t &key, int cap,
                                                   int &err, uint32_t bound) {
    const volatile uint64_t *vp = P;
    for (int i = 0; i < cap; ++i) {
        const uint64_t v = vp[s];
        const uint32_t p = (uint32_t)v;
        if (p == s) { key = (uint32_t)(v >> 32); return s; }
        if (p >= bound) break;
        s = p;
    }
    err |= kErrGlobalCap;
    key = 0xFFFFFFFFu;
    return s;
}

__device__ __forceinline__ void union_global(uint64_t *P, uint32_t a, uint32_t b, int cap, int &err,
                                             uint32_t bound) {
    for (int i = 0; i < cap; ++i) {
        uint32_t ka, kb;
        a = find_global(P, a, ka, cap, err, bound);
        b = find_global(P, b, kb, cap, err, bound);
        if (a == b || err) return;
        if (ka < kb) { uint32_t t = a; a = b; b = t; t = ka; ka = kb; kb = t; }
        const unsigned long long old =
            atomicMin((unsigned long long *)(P + a), (unsigned long long)pack_slot(kb, b));
        if (old == pack_slot(ka, a)) return;
        a = (uint32_t)old;
        if (a >= bound) break;
    }
    err |= kErrGlobalCap;
}

}  // namespace ccl
