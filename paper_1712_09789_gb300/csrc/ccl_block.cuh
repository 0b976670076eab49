// ccl_block.cuh -- device building blocks of the block-based labeller.
//
// Geometry.  A CTA owns a block of (32 * BLX) x (8 * BLY) pixels and has one
// thread per lane tile of 32 columns x 8 rows (tx = t % BLX, ty = t / BLX).
// A thread scans its lane tile row by row, holding each row as a 32-bit mask
// (bit c = column c).  The paper's Kernel 1 assigns one thread per pixel and
// iterates over the whole block; here one thread walks its rows in order,
// which makes the label-equivalence work proportional to the number of row
// runs, and BLX * BLY such walks run side by side.  The block shape (BLX, BLY)
// is a template parameter so that the batched path can pick it per workload.
//
// Label-equivalence lists.  Every lane tile numbers its own labels 0..127 in
// creation order (creation order is raster order inside the lane tile, so the
// smallest label of a list is also its smallest pixel).  A list entry is a
// 16-bit word in shared memory: a root holds kRoot | node, node = r*32 + c its
// first pixel; any other entry holds the id (t << 7) | label of its parent,
// which may belong to another lane tile once the tiles of a block are merged.
// Entry of id i lives at par[(i & 127) * threads + (i >> 7)], so the 32 lanes of
// a warp touching their own label L hit 32 consecutive half-words.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace ccl {

constexpr int kLW = 32;                 // lane tile width (bits of a row mask)
constexpr int kLH = 8;                  // lane tile height (rows walked by a thread)
constexpr int kLabCap = kLH * 16;       // labels per lane tile (<= 16 runs per row)
constexpr int kRunCap = kLH * 16;       // runs per lane tile
constexpr int kLWords = kRunCap / 4;    // 4 one-byte labels per 32-bit word
constexpr int kVChunks = kRunCap / 8;   // 8 two-byte values per 16-byte chunk
constexpr uint16_t kRoot = 0x8000;
constexpr uint16_t kRootBorder = 0x4000;
constexpr uint16_t kBg = 0xFFFF;
constexpr uint16_t kBorderFlag = 0x8000;  // per-run value: border slot, else block key
constexpr unsigned kFull = 0xFFFFFFFFu;

constexpr int kErrLocalCap = 1;
constexpr int kErrGlobalCap = 2;

constexpr int ilog2(int v) { return v <= 1 ? 0 : 1 + ilog2(v / 2); }

template <int BLX_, int BLY_>
struct Geo {
    static constexpr int BLX = BLX_;                  // lane tiles across a block
    static constexpr int BLY = BLY_;                  // lane tiles down a block
    static constexpr int kThreads = BLX * BLY;
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
    static constexpr int kLabPitch = kThreads + 4;    // bytes per column row of the label buffers
    // ids carry the thread index above 7 label bits and stay below kRootBorder;
    // block keys fit the 15 bits of a per-run value
    static_assert(kThreads >= 32 && kThreads <= 128 && (kThreads & (kThreads - 1)) == 0,
                  "32..128 threads, a power of two");
    static_assert((BLX & (BLX - 1)) == 0, "BLX must be a power of two");
    static_assert(kBW * kBH <= 32768, "block keys must fit 15 bits");
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

// Run mask of bits a0..a1.  a1 == 31 wraps 2u << 31 to 0, which still gives
// the bits a0..31.
__device__ __forceinline__ uint32_t run_bits(int a0, int a1) { return (2u << a1) - (1u << a0); }

// Columns of the neighbouring row that touch a run: the run itself, widened by
// one column on each side for 8-connectivity.
template <bool kConn8>
__device__ __forceinline__ uint32_t touch_range(uint32_t rm) {
    return kConn8 ? (rm | (rm << 1) | (rm >> 1)) : rm;
}

// ---------------------------------------------------------------------------
// Shared-memory label-equivalence lists of one block.

// (masked on both fields, so no entry value can address outside the table)
template <class G>
__device__ __forceinline__ int par_index(int id) {
    return (id & (kLabCap - 1)) * G::kThreads + ((id >> 7) & (G::kThreads - 1));
}

// Block raster key (row * block width + column) of a root, from its id and entry.
template <class G>
__device__ __forceinline__ int root_key(int id, uint16_t entry) {
    const int t = id >> 7;
    const int node = entry & 0xFF;
    return ((kLH * (t >> G::kBLXLog2) + (node >> 5)) << G::kBWLog2) + kLW * (t & (G::BLX - 1)) + (node & 31);
}

// Root of id and the root's entry.  Path halving rewrites only non-root
// entries, and links are only ever made on roots (by CAS), so the two never
// overwrite each other.
template <class G>
__device__ __forceinline__ int find_root(volatile uint16_t *par, int x, uint16_t &rentry, int cap, int &err) {
    for (int i = 0; i < cap; ++i) {
        const uint16_t e = par[par_index<G>(x)];
        if (e & kRoot) { rentry = e; return x; }
        const uint16_t g = par[par_index<G>(e)];
        if (g & kRoot) { rentry = g; return e; }
        par[par_index<G>(x)] = g;
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
template <class G>
__device__ __forceinline__ int find_root_ro(const volatile uint16_t *par, int x, int cap, int &err) {
    for (int i = 0; i < cap; ++i) {
        const uint16_t e = par[par_index<G>(x)];
        if (e & kRoot) return x;
        x = e;
    }
    err |= kErrLocalCap;
    return x;
}

// Merge the lists of ids a and b, called by all 32 lanes of a warp together
// (lanes with valid == false only keep step): the root with the larger key is
// hung under the root with the smaller key (Sec. 3.1.3 and 3.2: the larger
// label points to the smaller).  A failed CAS means the root changed
// meanwhile; the round repeats until no lane needs another, so the warp stays
// converged between rounds.
template <class G>
__device__ __forceinline__ void union_block_sync(uint16_t *par, bool valid, int a, int b, int cap, int &err) {
    volatile uint16_t *vp = par;
    bool pend = valid;
    for (int i = 0; __any_sync(kFull, pend); ++i) {
        if (pend) {
            uint16_t ea, eb;
            a = find_root<G>(vp, a, ea, cap, err);
            b = find_root<G>(vp, b, eb, cap, err);
            if (a == b || err) {
                pend = false;
            } else {
                if (root_key<G>(a, ea) < root_key<G>(b, eb)) {
                    const int t = a; a = b; b = t;
                    const uint16_t u = ea; ea = eb; eb = u;
                }
                const unsigned short old = atomicCAS(reinterpret_cast<unsigned short *>(par + par_index<G>(a)),
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

// After the lists of a block are final, root entries are rewritten as the
// value every run of that list needs later: kRootBorder | slot for a root
// that owns a block-border pixel, kRoot | block key otherwise; non-root
// entries then take their root's value.
template <class G>
__device__ __forceinline__ uint16_t run_value(const volatile uint16_t *par, int id) {
    uint16_t e = par[par_index<G>(id)];
    if (e < kRootBorder) e = par[par_index<G>(e)];
    // still a pointer only when an iteration cap cut the compression short
    // (the error word is set then); decode it as block key 0, never as a slot
    if (e < kRootBorder) return 0;
    return (e & kRoot) ? (uint16_t)(e & 0x7FFF) : (uint16_t)(kBorderFlag | (e & 0x3FFF));
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
