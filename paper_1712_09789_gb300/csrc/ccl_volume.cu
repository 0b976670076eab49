// ccl_volume.cu -- connected components of a 3D binary volume.
//
// Sec. 1 states the labelling task for 2D and 3D images; the paper works the
// method out in 2D.  This is the same coarse-to-fine structure one dimension
// up, on blocks of 32 x 16 x 16 voxels (one CTA, one thread per 32-voxel row
// held as a bit mask):
//   k_vol_local  step 1 (Sec. 3.1).  Under 6-connectivity the elements are
//                the runs of each row; coarse labelling gives each run its
//                first contact in an earlier row of the block (the row above,
//                the row in the slice before) as parent.  Under
//                26-connectivity the elements are the pieces of 2 x 2 row
//                bundles (runs of the OR of four rows, see Bundle), linked to
//                the four earlier bundles the same way.  The other contacts
//                are joined by a shared-memory union-find whose links go from
//                the larger block position to the smaller, so a root is its
//                component's first voxel in raster order.  Roots of
//                components that touch a neighbouring block's foreground get
//                a border slot and an entry of the global union-find over
//                slots, keyed by their global position (ID conversion, Sec.
//                3.1.4).  Outputs: the row masks, one 16-bit value per element
//                (border slot or block position of its root) and, for every
//                voxel of the six block faces, the slot of its root.
//   k_vol_merge  step 2 (Sec. 3.2): every voxel pair across a block face
//                joins its two slots in the global union-find (lock-free
//                atomicMin union, the pairs deduplicated per CTA); a pair
//                that crosses several faces is taken by the z face, else the
//                y face, else the x face, so each pair is seen once.
//   k_vol_write  step 3 (Sec. 3.3): the element index of every voxel is
//                rebuilt from the row masks, each element's value becomes its
//                final label (border slots by a root-find in the merged
//                union-find) and every voxel of the block is written once, as
//                whole 128-byte rows.
// Labels: 1 + min raster position x + y*W + z*W*H of the component, 0 for
// background.  Nothing but the final labels is written to `labels`.
#include <cstdint>

#include <cuda_runtime.h>

#include "ccl_block.cuh"
#include "ccl_internal.h"

namespace ccl {
namespace {

constexpr int kVX = 32, kVY = 16, kVZ = 16;  // block: voxels along x, y, z
constexpr int kVRows = kVY * kVZ;            // rows of 32 voxels per block
constexpr int kVThreads = kVRows;            // one thread per row
constexpr int kVIds = kVRows * kVX;          // ids: row * 32 + x (row = z * kVY + y)
constexpr int kPairHash = 2048;              // slot pairs remembered per CTA in the merge
constexpr unsigned long long kNoPair = ~0ull;
// Element values (one u16 per element, in element order): the block
// position (id) of the element's root, or kSlotFlag | border slot of that
// root when its component touches a neighbouring block.
constexpr uint16_t kSlotFlag = 0x8000;
// Elements per block at most: 16 runs in each row (6-connectivity), 16
// pieces in each of the 64 bundles (26-connectivity).
constexpr int kVMaxElems = kVRows * kVX / 2;
// Border slots per block at most: a border root's component holds a
// foreground voxel of a block face, so there are no more of them than face
// voxels.
constexpr int kVFaceVoxels = 2 * (kVY * kVX + kVZ * kVX + kVZ * kVY);
constexpr int kVSlots = kVFaceVoxels;
// Face records: for every voxel of the six faces, the border slot of its
// root, kNoSlot for background (and for a root without a slot, whose
// component meets no foreground across the face).  Per block:
//   [kFaceZ0 + y*32 + x]   slice z = 0       [kFaceZ1 + y*32 + x]  slice z = 15
//   [kFaceY0 + z*32 + x]   rows y = 0        [kFaceY1 + z*32 + x]  rows y = 15
//   [kFaceX0 + z*16 + y]   voxels x = 0      [kFaceX1 + z*16 + y]  voxels x = 31
constexpr uint16_t kNoSlot = 0xFFFF;
constexpr int kFaceZ0 = 0, kFaceZ1 = kVY * kVX, kFaceY0 = 2 * kVY * kVX, kFaceY1 = kFaceY0 + kVZ * kVX;
constexpr int kFaceX0 = kFaceY1 + kVZ * kVX, kFaceX1 = kFaceX0 + kVRows;
static_assert(kFaceX1 + kVRows == kVFaceVoxels, "face record layout");
static_assert(kVIds < kSlotFlag && kVSlots < kSlotFlag, "ids and slots must fit the element values");
static_assert(kVMaxElems < 65536 && kVSlots < 65536, "the step-1 scan packs both counts in 16 bits");

__device__ int g_volume_error = 0;

struct VolArgs {
    const uint8_t *img;
    int32_t *labels;
    uint32_t *mask;   // row masks, kVRows per block
    uint16_t *vals;   // element values, kVMaxElems per block (the first ones used)
    uint16_t *face;   // face records, kVFaceVoxels per block
    uint64_t *P;      // global union-find over border slots, kVSlots per block
    uint32_t *ns;     // border slots per block
    unsigned long long pitch;
    int D, H, W;
    int n;  // voxels, D * H * W
    int nbx, nby, nbz;
    int vec_in;
    int vec_out;  // labels rows start 16-byte aligned (W % 4 == 0, aligned base)
    int local_cap, global_cap;
    uint32_t bound;  // slots in all: blocks * kVSlots
};

constexpr int kCand = 2048;  // refinement pairs listed per pass (more are joined at once)

struct VolSmem {
    uint32_t mask[kVRows];    // row masks (bit x = voxel x of the row)
    uint32_t border[kVRows];  // bit x of row r: id r*32+x is a marked root (border slot owner)
    uint32_t par[kVIds];      // union-find entries, by slot(id); used at element ids only
    uint32_t cand[kCand];     // refinement pairs (a << 16 | b)
    uint32_t wtot[kVThreads / 32];
    unsigned ncand;
};

// Storage slot of an id: rows keep their 32 entries, rotated by the row so
// that threads on different rows touching the same column use other banks.
__device__ __forceinline__ int slot(int id) { return (id & ~31) | ((id + (id >> 5)) & 31); }

// Last voxel of the run of m that holds voxel b.
__device__ __forceinline__ int run_end(uint32_t m, int b) {
    const uint32_t z = ~m & (~0u << b);
    return z ? lobit(z) - 1 : 31;
}

__device__ __forceinline__ long long vpos(const VolArgs &a, int x, int y, int z) {
    return (long long)x + (long long)a.W * ((long long)y + (long long)a.H * z);
}

__device__ __forceinline__ int v_find(volatile uint32_t *par, int x, int cap, int &err) {
    for (int i = 0; i < cap; ++i) {
        const int p = (int)par[slot(x)];
        if (p == x) return x;
        const int q = (int)par[slot(p)];
        if (q == p) return p;
        par[slot(x)] = (uint32_t)q;  // halving: an ancestor, never loses a link
        x = q;
    }
    err |= kErrLocalCap;
    return x;
}

// Root of x with path halving by CAS: a halving store lands only while the
// entry still holds the parent the walk read, so it never overwrites the root
// that the entry's own thread stores meanwhile (the compression pass).
__device__ __forceinline__ int v_find_cas(uint32_t *par, int x, int cap, int &err) {
    volatile uint32_t *vp = par;
    for (int i = 0; i < cap; ++i) {
        const int p = (int)vp[slot(x)];
        if (p == x) return x;
        const int g = (int)vp[slot(p)];
        if (g == p) return p;
        atomicCAS(par + slot(x), (uint32_t)p, (uint32_t)g);
        x = g;
    }
    err |= kErrLocalCap;
    return x;
}

// Joins the sets of ids a and b; the larger root is hung under the smaller.
__device__ void v_union(uint32_t *par, int a, int b, int cap, int &err) {
    volatile uint32_t *vp = par;
    for (int i = 0; i < cap; ++i) {
        a = v_find(vp, a, cap, err);
        b = v_find(vp, b, cap, err);
        if (a == b || err) return;
        if (a < b) {
            const int t = a;
            a = b;
            b = t;
        }
        const int old = (int)atomicMin(par + slot(a), (uint32_t)b);
        if (old == a) return;
        a = old;  // a gained a parent meanwhile: join that one instead
    }
    err |= kErrLocalCap;
}

// Exclusive prefix sum of v over the CTA's kVThreads threads, in thread
// order; `total` gets the sum over all threads.  wtot holds kVThreads / 32
// words; the call ends with the barrier after which they may be reused.
__device__ __forceinline__ uint32_t cta_exclusive_scan(uint32_t v, uint32_t *wtot, uint32_t &total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t s = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t u = __shfl_up_sync(0xFFFFFFFFu, s, d);
        if (lane >= d) s += u;
    }
    if (lane == 31) wtot[warp] = s;
    __syncthreads();
    uint32_t base = 0, tot = 0;
#pragma unroll
    for (int w = 0; w < kVThreads / 32; ++w) {
        const uint32_t x = wtot[w];
        if (w < warp) base += x;
        tot += x;
    }
    total = tot;
    __syncthreads();
    return base + s - v;
}

// Two steps up from x: x itself for a root, else its parent's parent (its
// parent when that is a root).  Equal results mean one set.
__device__ __forceinline__ int v_root2(const volatile uint32_t *par, int x) {
    return (int)par[slot((int)par[slot(x)])];
}

// Joins the sets of a and b, by all 32 lanes of a warp together (lanes with
// valid == false keep step), with the links of v_union.
__device__ __forceinline__ void v_union_sync(uint32_t *par, bool valid, int a, int b, int cap, int &err) {
    volatile uint32_t *vp = par;
    bool pend = valid;
    for (int i = 0; __any_sync(0xFFFFFFFFu, pend); ++i) {
        if (pend) {
            a = v_find(vp, a, cap, err);
            b = v_find(vp, b, cap, err);
            if (a == b || err) {
                pend = false;
            } else {
                if (a < b) {
                    const int t = a;
                    a = b;
                    b = t;
                }
                const int old = (int)atomicMin(par + slot(a), (uint32_t)b);
                if (old == a) pend = false;
                else a = old;  // a gained a parent meanwhile: join that one instead
            }
        }
        if (i >= cap) {
            if (pend) err |= kErrLocalCap;
            break;
        }
    }
}

// A refinement pair (two element ids): listed for join_candidates, or
// joined at once when the list is full.
__device__ __forceinline__ void emit_pair(VolSmem &sm, int a, int b, int cap, int &err) {
    const unsigned i = atomicAdd(&sm.ncand, 1u);
    if (i < (unsigned)kCand) sm.cand[i] = ((uint32_t)a << 16) | (uint32_t)b;
    else v_union(sm.par, a, b, cap, err);
}

// After the barrier that follows the last emit_pair: every lane takes one
// listed pair per step and joins it where the two-step roots differ.
__device__ __forceinline__ void join_candidates(VolSmem &sm, int cap, int &err) {
    const unsigned nc = sm.ncand < (unsigned)kCand ? sm.ncand : (unsigned)kCand;
    for (unsigned j0 = 0; j0 < nc; j0 += kVThreads) {
        const unsigned j = j0 + threadIdx.x;
        int a = 0, b = 0;
        bool need = false;
        if (j < nc) {
            const uint32_t e = sm.cand[j];
            a = (int)(e >> 16);
            b = (int)(e & 0xFFFFu);
            need = v_root2(sm.par, a) != v_root2(sm.par, b);
        }
        v_union_sync(sm.par, need, a, b, cap, err);
    }
}

// Row (y, z) of the volume over the block's 32 columns from gx0, as a bit
// mask; rows outside the volume are empty.
__device__ __forceinline__ uint32_t row_mask(const VolArgs &a, int gx0, int gy, int gz) {
    if (gy < 0 || gz < 0 || gy >= a.H || gz >= a.D) return 0u;
    const uint8_t *p = a.img + ((size_t)gz * a.H + gy) * a.pitch + gx0;
    if (a.vec_in && gx0 + kVX <= a.W) {
        const uint4 lo = ldg_nc16(p), hi = ldg_nc16(p + 16);
        return nz16(lo) | (nz16(hi) << 16);
    }
    uint32_t m = 0;
    const int n = a.W - gx0 < kVX ? a.W - gx0 : kVX;
    for (int i = 0; i < n; ++i) m |= (uint32_t)(__ldg(p + i) != 0) << i;
    return m;
}

// 26-connectivity works on bundles of 2 x 2 rows: (2Y, 2Z), (2Y+1, 2Z),
// (2Y, 2Z+1), (2Y+1, 2Z+1).  Every voxel of a bundle column touches every
// voxel of the same and the two neighbouring columns of the bundle (|dx|,
// |dy|, |dz| <= 1), so the components inside a bundle are the runs of the OR
// of its four rows ("pieces"), found by bit operations.  A piece is named by
// its first voxel in raster order: the first of the four rows it occupies
// (they are in increasing id order), first column there.  A piece name is a
// voxel id, so the union-find over pieces keeps the order of voxel ids.
struct Bundle {
    uint32_t m0, m1, m2, m3;  // rows r0, r0 + 1, r0 + kVY, r0 + kVY + 1
    int r0;
};

__device__ __forceinline__ int bundle_row0(int r) { return (r / kVY & ~1) * kVY + (r % kVY & ~1); }

__device__ __forceinline__ Bundle load_bundle(const VolSmem &sm, int r0) {
    return {sm.mask[r0], sm.mask[r0 + 1], sm.mask[r0 + kVY], sm.mask[r0 + kVY + 1], r0};
}

__device__ __forceinline__ uint32_t bundle_or(const Bundle &b) { return b.m0 | b.m1 | b.m2 | b.m3; }

__device__ __forceinline__ int piece_key(const Bundle &b, int s, int e) {
    const uint32_t rb = run_bits(s, e);
    if (b.m0 & rb) return b.r0 * kVX + lobit(b.m0 & rb);
    if (b.m1 & rb) return (b.r0 + 1) * kVX + lobit(b.m1 & rb);
    if (b.m2 & rb) return (b.r0 + kVY) * kVX + lobit(b.m2 & rb);
    return (b.r0 + kVY + 1) * kVX + lobit(b.m3 & rb);
}

// Name of the piece that holds voxel x (x must be in the bundle's OR).
__device__ __forceinline__ int piece_key_at(const Bundle &b, int x) {
    const uint32_t o = bundle_or(b);
    return piece_key(b, hibit(o & ~(o << 1) & upto(x)), run_end(o, x));
}

// The earlier bundles a bundle (Y, Z) can touch, in the order they are
// visited, and which rows of each side face the other:
//   0: (Y-1, Z)    own rows y = 2Y      vs its rows y = 2Y-1
//   1: (Y, Z-1)    own rows z = 2Z      vs its rows z = 2Z-1
//   2: (Y-1, Z-1)  own row (2Y, 2Z)     vs its row (2Y-1, 2Z-1)
//   3: (Y+1, Z-1)  own row (2Y+1, 2Z)   vs its row (2Y+2, 2Z-1)
__device__ __forceinline__ int bundle_nb_off(int k) {
    return k == 0 ? -2 : k == 1 ? -2 * kVY : k == 2 ? -2 * kVY - 2 : -2 * kVY + 2;
}
__device__ __forceinline__ uint32_t bundle_own_face(const Bundle &b, int k) {
    return k == 0 ? (b.m0 | b.m2) : k == 1 ? (b.m0 | b.m1) : k == 2 ? b.m0 : b.m1;
}
__device__ __forceinline__ uint32_t bundle_nb_face(const Bundle &n, int k) {
    return k == 0 ? (n.m1 | n.m3) : k == 1 ? (n.m2 | n.m3) : k == 2 ? n.m3 : n.m2;
}

// Root of voxel x of row r once the block's lists are compressed.
template <bool k26>
__device__ __forceinline__ int voxel_root(const VolSmem &sm, int r, int x) {
    if (k26) return (int)sm.par[slot(piece_key_at(load_bundle(sm, bundle_row0(r)), x))];
    const uint32_t mr = sm.mask[r];
    return (int)sm.par[slot(r * kVX + hibit(mr & ~(mr << 1) & upto(x)))];
}

// Step 1 for 26-connectivity on the block's 64 bundles.  Thread t works on
// bundle t % 64: in the contact pass against the earlier bundle k = t / 64,
// in the per-piece passes on every fourth piece of the bundle from k on.
// Column connection: each contact of a piece with a piece of a smaller name
// lowers the piece's entry to that name (atomicMin: the entry ends at the
// smallest such neighbour, so the links go to smaller names and form a
// forest).  Refinement: every contact is also listed as a pair (those that
// made a link are dropped by the root filter of join_candidates).
// Compression follows.  Ends with a barrier.
__device__ void bundle_labelling(VolSmem &sm, const VolArgs &a, int &err) {
    constexpr int kBY = kVY / 2, kBZ = kVZ / 2;
    static_assert(kBY * kBZ * 4 == kVThreads, "one thread per bundle and earlier bundle");
    const int t = threadIdx.x;
    const int bt = t % (kBY * kBZ), k = t / (kBY * kBZ);
    const int Yb = bt % kBY, Zb = bt / kBY;
    const int rb = 2 * Zb * kVY + 2 * Yb;
    const Bundle bb = load_bundle(sm, rb);
    const uint32_t ob = bundle_or(bb), starts = ob & ~(ob << 1);
    {
        int j = 0;
        for (uint32_t q = starts; q; q &= q - 1, ++j) {
            if ((j & 3) != k) continue;
            const int s = lobit(q);
            const int key = piece_key(bb, s, run_end(ob, s));
            sm.par[slot(key)] = (uint32_t)key;
        }
    }
    __syncthreads();
    const bool on = k == 0 ? Yb > 0 : k == 1 ? Zb > 0 : k == 2 ? (Yb > 0 && Zb > 0) : (Yb < kBY - 1 && Zb > 0);
    Bundle n = {0u, 0u, 0u, 0u, 0};
    uint32_t no = 0, fo = 0, fn = 0;
    if (on) {
        n = load_bundle(sm, rb + bundle_nb_off(k));
        no = bundle_or(n);
        fo = bundle_own_face(bb, k);
        fn = bundle_nb_face(n, k);
        if (!(touch_range<true>(fo) & fn)) fo = 0;
    }
    // the contacts of the own pieces with the pieces of bundle n: one per
    // (piece, piece) pair
    const auto contacts = [&](auto &&visit) {
        if (!fo) return;
        for (uint32_t q = starts; q; q &= q - 1) {
            const int s = lobit(q), e = run_end(ob, s);
            uint32_t c = touch_range<true>(fo & run_bits(s, e)) & fn;
            if (!c) continue;
            const int key = piece_key(bb, s, e);
            while (c) {
                const int bit = lobit(c);
                visit(key, piece_key_at(n, bit));
                const int ne = run_end(no, bit);
                c = ne == 31 ? 0u : c & (~0u << (ne + 1));
            }
        }
    };
    contacts([&](int key, int nk) {
        if (nk < key) atomicMin(&sm.par[slot(key)], (uint32_t)nk);
        const unsigned i = atomicAdd(&sm.ncand, 1u);
        if (i < (unsigned)kCand) sm.cand[i] = ((uint32_t)key << 16) | (uint32_t)nk;
    });
    __syncthreads();
    join_candidates(sm, a.local_cap, err);
    if (sm.ncand > (unsigned)kCand) {
        // the list overflowed: every contact is joined once more, one by one
        __syncthreads();
        contacts([&](int key, int nk) { v_union(sm.par, key, nk, a.local_cap, err); });
    }
    __syncthreads();
    {
        int j = 0;
        for (uint32_t q = starts; q; q &= q - 1, ++j) {
            if ((j & 3) != k) continue;
            const int s = lobit(q);
            const int key = piece_key(bb, s, run_end(ob, s));
            const int root = v_find_cas(sm.par, key, a.local_cap, err);
            if (root != key) sm.par[slot(key)] = (uint32_t)root;
        }
    }
    __syncthreads();
}

// Step 1 inside the block (bx, by, bz): masks, runs, unions, compression and
// the border-root marks.  Ends with a barrier; the thread's row mask is
// returned.
template <bool k26>
__device__ uint32_t vol_local(VolSmem &sm, const VolArgs &a, int bx, int by, int bz, int &err) {
    const int r = threadIdx.x, y = r % kVY, z = r / kVY;
    const int gx0 = bx * kVX, gy = by * kVY + y, gz = bz * kVZ + z;
    const uint32_t m = row_mask(a, gx0, gy, gz);

    // Voxels of this row that may touch a foreground voxel of a neighbouring
    // block: only their components need a border slot.  Under
    // 6-connectivity a voxel of a y or z face counts when the voxel across
    // it is foreground (the row across is read); under 26-connectivity every
    // voxel of a face row counts.  The x faces count wherever the edge
    // voxel is foreground.
    uint32_t across = 0;
    {
        const bool fy0 = y == 0 && by > 0, fy1 = y == kVY - 1 && by < a.nby - 1;
        const bool fz0 = z == 0 && bz > 0, fz1 = z == kVZ - 1 && bz < a.nbz - 1;
        if (k26) {
            // a voxel of a y or z face meets nine voxels across it, and one
            // of them is nearly always foreground: every voxel of such a row
            // counts (no reads across the face)
            if (fy0 || fy1 || fz0 || fz1) across = ~0u;
        } else {
            // (the loads go out together with the own row's)
            if (fy0) across |= row_mask(a, gx0, gy - 1, gz);
            if (fy1) across |= row_mask(a, gx0, gy + 1, gz);
            if (fz0) across |= row_mask(a, gx0, gy, gz - 1);
            if (fz1) across |= row_mask(a, gx0, gy, gz + 1);
        }
        across |= (bx > 0 ? 1u : 0u) | (bx < a.nbx - 1 ? 0x80000000u : 0u);
    }
    sm.mask[r] = m;
    sm.border[r] = 0;
    if (r == 0) sm.ncand = 0;
    __syncthreads();

    if (k26) {
        bundle_labelling(sm, a, err);
    } else {
        const uint32_t st = m & ~(m << 1);
        // contact events with the row above (u) and the row of the slice
        // before (v): a run of m & m_u lies inside one (run, run) pair, so
        // its first column is one event per pair
        const uint32_t mu = y > 0 ? sm.mask[r - 1] : 0u, mv = z > 0 ? sm.mask[r - kVY] : 0u;
        const uint32_t cu = m & mu, cv = m & mv;
        const uint32_t eu = cu & ~(cu << 1), ev = cv & ~(cv << 1);
        // coarse labelling: the lowest event of each run (the one with the
        // row above where both rows have one in that column) makes the run it
        // meets, of an earlier row and so of a smaller id, the run's parent;
        // a run without events is a root.  Only the own entries are written.
        const uint32_t e = eu | ev;
        const uint32_t fe = ((m + e) ^ m) & e;  // lowest event of every run
        for (uint32_t t = st; t; t &= t - 1) {
            const int s = lobit(t), id = r * kVX + s;
            const uint32_t f = fe & run_bits(s, run_end(m, s));
            int parent = id;
            if (f) {
                const int c = lobit(f);
                const bool up = (eu >> c) & 1u;
                const uint32_t mn = up ? mu : mv;
                parent = (r - (up ? 1 : kVY)) * kVX + hibit(mn & ~(mn << 1) & upto(c));
            }
            sm.par[slot(id)] = (uint32_t)parent;
        }
        __syncthreads();
        // one round of pointer jumping: every link to its grandparent (an
        // ancestor either way when another thread's store races with the
        // read), halving the chains of coarse links up the rows
        for (uint32_t t = st; t; t &= t - 1) {
            const int id = r * kVX + lobit(t);
            const uint32_t p = sm.par[slot(id)];
            if (p != (uint32_t)id) sm.par[slot(id)] = sm.par[slot((int)p)];
        }
        __syncthreads();

        // refinement: every other event joins its two runs
        const uint32_t su = mu & ~(mu << 1), sv = mv & ~(mv << 1);
        for (uint32_t t = eu & ~fe; t; t &= t - 1) {
            const int c = lobit(t);
            emit_pair(sm, r * kVX + hibit(st & upto(c)), (r - 1) * kVX + hibit(su & upto(c)), a.local_cap, err);
        }
        for (uint32_t t = ev & ~(fe & ~eu); t; t &= t - 1) {
            const int c = lobit(t);
            emit_pair(sm, r * kVX + hibit(st & upto(c)), (r - kVY) * kVX + hibit(sv & upto(c)), a.local_cap, err);
        }
        __syncthreads();
        join_candidates(sm, a.local_cap, err);
        __syncthreads();

        for (uint32_t t = st; t; t &= t - 1) {
            const int id = r * kVX + lobit(t);
            const int root = v_find_cas(sm.par, id, a.local_cap, err);
            if (root != id) sm.par[slot(id)] = (uint32_t)root;
        }
        __syncthreads();
    }

    // roots of the components with a voxel that may touch a neighbouring block
    uint32_t fm = m & across;
    while (fm) {
        const int b = lobit(fm);
        const int root = voxel_root<k26>(sm, r, b);
        atomicOr(&sm.border[root / kVX], 1u << (root % kVX));
        const int e = run_end(m, b);
        fm = e == 31 ? 0u : fm & (~0u << (e + 1));
    }
    __syncthreads();
    return m;
}

__device__ __forceinline__ void block_coords(const VolArgs &a, int &bx, int &by, int &bz) {
    const int b = blockIdx.x;
    bx = b % a.nbx;
    by = (b / a.nbx) % a.nby;
    bz = b / (a.nbx * a.nby);
}

// Element starts of thread t: the run starts of its row (6-connectivity),
// the piece starts of bundle t (26-connectivity, threads 0..63).  Elements
// are numbered thread after thread, start after start; *o gets the mask the
// starts belong to (the row, or the bundle's OR).
template <bool k26>
__device__ __forceinline__ uint32_t element_starts(const uint32_t *mask, int t, uint32_t &o, int &r0) {
    if (k26) {
        constexpr int kBY = kVY / 2, kBZ = kVZ / 2;
        r0 = 2 * (t / kBY) * kVY + 2 * (t % kBY);
        o = t < kBY * kBZ ? (mask[r0] | mask[r0 + 1] | mask[r0 + kVY] | mask[r0 + kVY + 1]) : 0u;
    } else {
        r0 = t;
        o = mask[t];
    }
    return o & ~(o << 1);
}

template <bool k26>
__global__ void __launch_bounds__(kVThreads, 5) k_vol_local(VolArgs a) {
    __shared__ VolSmem sm;
    __shared__ uint16_t sbase[kVRows];      // border slot of the first marked root of each row
    __shared__ uint16_t eoff[kVThreads];    // first element of each thread's row (bundle)
    // the merge may be launched once every CTA of this grid has started (it
    // waits for this grid's completion before reading anything)
    grid_launch_dependents();
    int bx, by, bz;
    block_coords(a, bx, by, bz);
    int err = 0;
    const uint32_t m = vol_local<k26>(sm, a, bx, by, bz, err);
    const int r = threadIdx.x, y = r % kVY, z = r / kVY;
    const int gx0 = bx * kVX, gy0 = by * kVY, gz0 = bz * kVZ;
    const size_t b = blockIdx.x;

    // border slots of the marked roots and element numbers, by one scan of
    // both counts (16 bits each)
    uint32_t o;
    int r0;
    const uint32_t est = element_starts<k26>(sm.mask, r, o, r0);
    const uint32_t bd = sm.border[r];
    uint32_t tot;
    const uint32_t pre = cta_exclusive_scan((uint32_t)__popc(est) | ((uint32_t)__popc(bd) << 16), sm.wtot, tot);
    sbase[r] = (uint16_t)(pre >> 16);
    eoff[r] = (uint16_t)(pre & 0xFFFFu);
    if (r == 0) a.ns[b] = tot >> 16;
    a.mask[b * kVRows + r] = m;
    __syncthreads();
    const auto value_of = [&](int root) -> uint16_t {
        const int rr = root >> 5;
        const uint32_t bw = sm.border[rr];
        if (!((bw >> (root & 31)) & 1u)) return (uint16_t)root;
        return (uint16_t)(kSlotFlag | (sbase[rr] + __popc(bw & ((1u << (root & 31)) - 1u))));
    };

    // global union-find entries of the own row's border roots, keyed by the
    // root's global position (its component's first voxel in the block)
    {
        const uint32_t s0 = (uint32_t)(b * kVSlots) + (pre >> 16);
        uint32_t k = 0;
        for (uint32_t t = bd; t; t &= t - 1, ++k) {
            const uint32_t key = (uint32_t)vpos(a, gx0 + lobit(t), gy0 + y, gz0 + z);
            a.P[s0 + k] = pack_slot(key, s0 + k);
        }
    }
    // element values, staged in shared memory (the candidate list is free
    // now): the runs of the own row, or every fourth piece of bundle t % 64
    static_assert(sizeof(sm.cand) == kVMaxElems * sizeof(uint16_t), "the value stage fills the candidate list");
    uint16_t *const stage = reinterpret_cast<uint16_t *>(sm.cand);
    if (k26) {
        constexpr int kB = (kVY / 2) * (kVZ / 2);
        const int bt = r % kB, k = r / kB;
        const int rb = 2 * (bt / (kVY / 2)) * kVY + 2 * (bt % (kVY / 2));
        const Bundle bu = load_bundle(sm, rb);
        const uint32_t ob = bundle_or(bu);
        int j = 0;
        for (uint32_t t = ob & ~(ob << 1); t; t &= t - 1, ++j) {
            if ((j & 3) != k) continue;
            const int s = lobit(t);
            stage[eoff[bt] + j] = value_of((int)sm.par[slot(piece_key(bu, s, run_end(ob, s)))]);
        }
    } else {
        int e = eoff[r];
        for (uint32_t t = est; t; t &= t - 1, ++e) stage[e] = value_of((int)sm.par[slot(r * kVX + lobit(t))]);
    }
    __syncthreads();
    {
        const uint4 *src = reinterpret_cast<const uint4 *>(stage);
        uint4 *dst = reinterpret_cast<uint4 *>(a.vals + b * kVMaxElems);
        for (int i = r; i < (int)((tot & 0xFFFFu) + 7) / 8; i += kVThreads) dst[i] = src[i];
    }
    // face records from the staged values: the slices z = 0 and 15 and the
    // rows y = 0 and 15 one warp per row (lane = x), the voxels x = 0 and 31
    // of the own row
    uint16_t *F = a.face + b * kVFaceVoxels;
    const auto face_slot = [&](int row, int x) -> uint16_t {
        if (!((sm.mask[row] >> x) & 1u)) return kNoSlot;
        uint32_t st;
        int e0;
        if (k26) {
            const int rb = (row / kVY & ~1) * kVY + (row % kVY & ~1);
            const uint32_t ob = sm.mask[rb] | sm.mask[rb + 1] | sm.mask[rb + kVY] | sm.mask[rb + kVY + 1];
            st = ob & ~(ob << 1);
            e0 = eoff[(row / kVY / 2) * (kVY / 2) + (row % kVY) / 2];
        } else {
            const uint32_t mr = sm.mask[row];
            st = mr & ~(mr << 1);
            e0 = eoff[row];
        }
        const uint16_t v = stage[e0 + __popc(st & upto(x)) - 1];
        return (v & kSlotFlag) ? (uint16_t)(v & ~kSlotFlag) : kNoSlot;
    };
    {
        const int lane = r & 31, warp = r >> 5;
        for (int j = warp; j < 4 * 16; j += kVThreads / 32) {
            const int f = j >> 4, i = j & 15;
            const int row = f == 0 ? i : f == 1 ? (kVZ - 1) * kVY + i : f == 2 ? i * kVY : i * kVY + kVY - 1;
            F[f * (kVY * kVX) + i * kVX + lane] = face_slot(row, lane);
        }
    }
    F[kFaceX0 + r] = face_slot(r, 0);
    F[kFaceX1 + r] = face_slot(r, kVX - 1);
    if (err) atomicOr(&g_volume_error, err);
}

template <bool k26>
__global__ void __launch_bounds__(kVThreads) k_vol_merge(VolArgs a) {
    int bx, by, bz;
    block_coords(a, bx, by, bz);
    const int gx0 = bx * kVX, gy0 = by * kVY, gz0 = bz * kVZ;
    const uint32_t b = blockIdx.x;
    const uint16_t *own = a.face + (size_t)b * kVFaceVoxels;
    constexpr int kR = k26 ? 1 : 0;
    // slot pairs already joined by this CTA: most face voxels of a component
    // repeat the pair of their neighbours
    __shared__ unsigned long long seen[kPairHash];
    for (int i = threadIdx.x; i < kPairHash; i += kVThreads) seen[i] = kNoPair;
    // launched behind step 1 (programmatic dependent launch): wait for it,
    // then let the write-out start its prologue
    grid_dependency_wait();
    grid_launch_dependents();
    __syncthreads();
    int err = 0;
    uint32_t last_q = ~0u, last_p = ~0u;
    auto join = [&](uint32_t q, uint32_t p) {
        if (q == last_q && p == last_p) return;
        last_q = q;
        last_p = p;
        const unsigned long long key = ((unsigned long long)q << 32) | p;
        unsigned h = (unsigned)((key * 0x9E3779B97F4A7C15ull) >> 40) & (kPairHash - 1);
        for (int i = 0; i < 16; ++i, h = (h + 1) & (kPairHash - 1)) {
            unsigned long long cur = ((volatile unsigned long long *)seen)[h];
            if (cur == kNoPair) cur = atomicCAS(&seen[h], kNoPair, key);
            if (cur == key) return;      // joined by another thread of the CTA
            if (cur == kNoPair) break;   // claimed: this thread joins it
        }
        union_global(a.P, q, p, a.global_cap, err, a.bound);
    };
    const auto gslot = [](uint32_t blk, int k) { return blk * (uint32_t)kVSlots + (uint32_t)k; };
    // z face: own slice 0 against the last slice of the blocks below
    if (bz > 0) {
        for (int e = threadIdx.x; e < kVY * kVX; e += kVThreads) {
            const int q = own[kFaceZ0 + e];  // e = y * 32 + x
            if (q == kNoSlot) continue;
            const int gx = gx0 + e % kVX, gy = gy0 + e / kVX;
            for (int dy = -kR; dy <= kR; ++dy) {
                for (int dx = -kR; dx <= kR; ++dx) {
                    const int nx = gx + dx, ny = gy + dy;
                    if (nx < 0 || ny < 0 || nx >= a.W || ny >= a.H) continue;
                    const uint32_t nb = (uint32_t)(((bz - 1) * a.nby + ny / kVY) * a.nbx + nx / kVX);
                    const int p = a.face[(size_t)nb * kVFaceVoxels + kFaceZ1 + (ny % kVY) * kVX + nx % kVX];
                    if (p != kNoSlot) join(gslot(b, q), gslot(nb, p));
                }
            }
        }
    }
    // y face: own rows y = 0 against the rows y = 15 of the blocks in front,
    // in the same z block
    if (by > 0) {
        for (int e = threadIdx.x; e < kVZ * kVX; e += kVThreads) {
            const int q = own[kFaceY0 + e];  // e = z * 32 + x
            if (q == kNoSlot) continue;
            const int z = e / kVX, gx = gx0 + e % kVX;
            for (int dz = -kR; dz <= kR; ++dz) {
                const int zz = z + dz;
                if (zz < 0 || zz >= kVZ || gz0 + zz >= a.D) continue;
                for (int dx = -kR; dx <= kR; ++dx) {
                    const int nx = gx + dx;
                    if (nx < 0 || nx >= a.W) continue;
                    const uint32_t nb = (uint32_t)((bz * a.nby + by - 1) * a.nbx + nx / kVX);
                    const int p = a.face[(size_t)nb * kVFaceVoxels + kFaceY1 + zz * kVX + nx % kVX];
                    if (p != kNoSlot) join(gslot(b, q), gslot(nb, p));
                }
            }
        }
    }
    // x face: own voxels x = 0 against the voxels x = 31 of the block to the
    // left, in the same y and z block
    if (bx > 0) {
        const uint16_t *nf = a.face + (size_t)(b - 1) * kVFaceVoxels;
        for (int r = threadIdx.x; r < kVRows; r += kVThreads) {
            const int q = own[kFaceX0 + r];
            if (q == kNoSlot) continue;
            const int y = r % kVY, z = r / kVY;
            for (int dz = -kR; dz <= kR; ++dz) {
                const int zz = z + dz;
                if (zz < 0 || zz >= kVZ || gz0 + zz >= a.D) continue;
                for (int dy = -kR; dy <= kR; ++dy) {
                    const int yy = y + dy;
                    if (yy < 0 || yy >= kVY || gy0 + yy >= a.H) continue;
                    const int p = nf[kFaceX1 + zz * kVY + yy];
                    if (p != kNoSlot) join(gslot(b, q), gslot(b - 1, p));
                }
            }
        }
    }
    if (err) atomicOr(&g_volume_error, err);
}

// Step 3: the element index of every voxel from the row masks, the final
// label of every element (border slots through a root-find in the merged
// union-find), then every voxel of the block written once.
template <bool k26>
__global__ void __launch_bounds__(kVThreads) k_vol_write(VolArgs a) {
    __shared__ uint32_t mask[kVRows];
    __shared__ uint16_t eoff[kVThreads];  // first element of each thread's row or bundle
    __shared__ uint32_t wtot[kVThreads / 32];
    __shared__ int fin[kVSlots];          // final label by border slot
    __shared__ int lab[kVMaxElems];       // final label by element
    int bx, by, bz;
    block_coords(a, bx, by, bz);
    const int gx0 = bx * kVX, gy0 = by * kVY, gz0 = bz * kVZ;
    const size_t b = blockIdx.x;
    const int t = threadIdx.x;
    mask[t] = a.mask[b * kVRows + t];
    __syncthreads();
    uint32_t o, tot;
    int r0;
    const uint32_t est = element_starts<k26>(mask, t, o, r0);
    eoff[t] = (uint16_t)cta_exclusive_scan((uint32_t)__popc(est), wtot, tot);
    const int ns = (int)a.ns[b];
    // step 1's outputs are complete when this grid starts (the merge it runs
    // behind waited for step 1): the labels of the elements whose root has
    // no border slot are final now; a border slot s is held as -(s + 1)
    // positions in 32 bits: every voxel of the volume lies below 2^31
    const uint32_t W = (uint32_t)a.W, WH = W * (uint32_t)a.H;
    const uint32_t base = (uint32_t)gz0 * WH + (uint32_t)gy0 * W + (uint32_t)gx0;
    const uint16_t *V = a.vals + b * kVMaxElems;
    for (int e = t; e < (int)tot; e += kVThreads) {
        const int v = V[e];
        if (v & kSlotFlag) {
            lab[e] = -((v & ~kSlotFlag) + 1);
        } else {
            const uint32_t row = (uint32_t)v / kVX;
            lab[e] = (int)(base + (row / kVY) * WH + (row % kVY) * W + (uint32_t)v % kVX) + 1;
        }
    }
    // the merge (step 2) may still be running: wait for it before the first
    // read of the merged union-find
    grid_dependency_wait();
    int err = 0;
    for (int k = t; k < ns; k += kVThreads) {
        uint32_t key;
        find_global_ro(a.P, (uint32_t)(b * kVSlots) + (uint32_t)k, key, a.global_cap, err, a.bound);
        fin[k] = (int)key + 1;
    }
    __syncthreads();
    for (int e = t; e < (int)tot; e += kVThreads) {
        const int l = lab[e];
        if (l < 0) lab[e] = -l - 1 < ns ? fin[-l - 1] : 0;
    }
    __syncthreads();

    // whole rows: a lane takes 4 voxels (one 16-byte store), a warp 4 rows
    // per step; a lane keeps its y and steps two slices at a time
    const int lane = t % 32, warp = t / 32;
    const int c0 = 4 * (lane & 7);
    const int gx = gx0 + c0;
    const int row0 = 4 * warp + (lane >> 3);
    constexpr int kRowStep = 4 * (kVThreads / 32);
    static_assert(kRowStep % kVY == 0, "a lane's rows share their y");
    const int yl = row0 % kVY, gy = gy0 + yl;
    if (gy < a.H && gx < a.W) {
        const bool vec = a.vec_out && gx + 4 <= a.W;
        const int nx = a.W - gx < 4 ? a.W - gx : 4;
        const uint32_t pstep = (uint32_t)(kRowStep / kVY) * WH;
        uint32_t pos = base + (uint32_t)(row0 / kVY) * WH + (uint32_t)yl * W + (uint32_t)c0;
        for (int row = row0; row < kVRows && gz0 + row / kVY < a.D; row += kRowStep, pos += pstep) {
            const uint32_t m = mask[row];
            int v[4] = {0, 0, 0, 0};
            if ((m >> c0) & 15u) {
                uint32_t st;
                int e;
                if (k26) {
                    const int r0 = (row / kVY & ~1) * kVY + (yl & ~1);
                    const uint32_t o = mask[r0] | mask[r0 + 1] | mask[r0 + kVY] | mask[r0 + kVY + 1];
                    st = o & ~(o << 1);
                    e = (int)eoff[(row / kVY / 2) * (kVY / 2) + yl / 2];
                } else {
                    st = m & ~(m << 1);
                    e = (int)eoff[row];
                }
                e += __popc(st & ((1u << c0) - 1u)) - 1;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    e += (int)((st >> (c0 + j)) & 1u);
                    if ((m >> (c0 + j)) & 1u) v[j] = lab[e];
                }
            }
            int32_t *dst = a.labels + pos;
            if (vec) {
                __stcs(reinterpret_cast<int4 *>(dst), make_int4(v[0], v[1], v[2], v[3]));
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (j < nx) __stcs(dst + j, v[j]);
            }
        }
    }
    if (err) atomicOr(&g_volume_error, err);
}

void volume_grid(int D, int H, int W, int &nbx, int &nby, int &nbz) {
    nbx = (W + kVX - 1) / kVX;
    nby = (H + kVY - 1) / kVY;
    nbz = (D + kVZ - 1) / kVZ;
}

}  // namespace

namespace {

// Workspace layout, array after array, each 256-byte aligned: row masks,
// element values, face records, global union-find entries, slot counts.
struct VolLayout {
    size_t mask, vals, face, P, ns, bytes;
};

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

VolLayout volume_layout(size_t blocks) {
    VolLayout l;
    l.mask = 0;
    l.vals = align256(l.mask + blocks * kVRows * sizeof(uint32_t));
    l.face = align256(l.vals + blocks * kVMaxElems * sizeof(uint16_t));
    l.P = align256(l.face + blocks * kVFaceVoxels * sizeof(uint16_t));
    l.ns = align256(l.P + blocks * kVSlots * sizeof(uint64_t));
    l.bytes = align256(l.ns + blocks * sizeof(uint32_t));
    return l;
}

}  // namespace

size_t volume_workspace_bytes(int D, int H, int W) {
    int nbx, nby, nbz;
    volume_grid(D, H, W, nbx, nby, nbz);
    return volume_layout((size_t)nbx * nby * nbz).bytes;
}

int launch_volume(const uint8_t *img, int D, int H, int W, size_t pitch, int conn, int32_t *labels, void *ws,
                  cudaStream_t stream, int cap) {
    VolArgs a;
    a.img = img;
    a.labels = labels;
    a.pitch = pitch;
    a.D = D;
    a.H = H;
    a.W = W;
    a.n = (int)((long long)D * H * W);
    volume_grid(D, H, W, a.nbx, a.nby, a.nbz);
    const size_t nblocks = (size_t)a.nbx * a.nby * a.nbz;
    if (nblocks * kVSlots >= 0xFFFFFFFFull) return -1;  // slot numbers are 32-bit
    const VolLayout l = volume_layout(nblocks);
    unsigned char *w = static_cast<unsigned char *>(ws);
    a.mask = reinterpret_cast<uint32_t *>(w + l.mask);
    a.vals = reinterpret_cast<uint16_t *>(w + l.vals);
    a.face = reinterpret_cast<uint16_t *>(w + l.face);
    a.P = reinterpret_cast<uint64_t *>(w + l.P);
    a.ns = reinterpret_cast<uint32_t *>(w + l.ns);
    a.bound = (uint32_t)(nblocks * kVSlots);
    a.vec_in = (pitch % 16 == 0) && (reinterpret_cast<uintptr_t>(img) % 16 == 0);
    a.vec_out = (W % 4 == 0) && (reinterpret_cast<uintptr_t>(labels) % 16 == 0);
    // a find walks a strictly decreasing chain and a union retry strictly
    // lowers its node, so neither can take more steps than there are nodes
    const long long n = (long long)D * H * W;
    a.local_cap = cap > 0 ? cap : kVIds + 16;
    a.global_cap = cap > 0 ? cap : (int)(n + 16 < (1LL << 30) ? n + 16 : (1LL << 30));
    const unsigned blocks = (unsigned)nblocks;
    // step 1 is a plain launch: it overwrites the scratch that the previous
    // call's write-out reads.  The merge and the write-out may start while
    // the kernel before them drains (programmatic dependent launch); each
    // waits for it before reading what it wrote.
    const auto pdl = [&](void (*kernel)(VolArgs)) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(blocks);
        cfg.blockDim = dim3(kVThreads);
        cfg.stream = stream;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        return cudaLaunchKernelEx(&cfg, kernel, a) == cudaSuccess;
    };
    bool ok;
    if (conn == 26) {
        k_vol_local<true><<<blocks, kVThreads, 0, stream>>>(a);
        ok = cudaGetLastError() == cudaSuccess && pdl(k_vol_merge<true>) && pdl(k_vol_write<true>);
    } else {
        k_vol_local<false><<<blocks, kVThreads, 0, stream>>>(a);
        ok = cudaGetLastError() == cudaSuccess && pdl(k_vol_merge<false>) && pdl(k_vol_write<false>);
    }
    return ok ? 0 : -1;
}

int read_and_clear_volume_error(int *value) {
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_volume_error, sizeof(int)) != cudaSuccess) return -1;
    if (v) {
        const int zero = 0;
        if (cudaMemcpyToSymbol(g_volume_error, &zero, sizeof(int)) != cudaSuccess) return -1;
    }
    *value = v;
    return 0;
}

}  // namespace ccl
