// ccl_kernels.cu -- the steps of the block-based labeller as sm_103a kernels,
// and the launchers that enqueue them on a stream.
//
//   k_block_local   step 1, Kernel 1 (Sec. 3.1) on blocks of 32*BLX x kLH*BLY
//                   pixels.  Every thread labels its 32 x kLH lane tile band by
//                   band: coarse labelling hangs each piece under the first
//                   piece of the band above that it touches (row connection
//                   is free inside a piece; column connection by bit
//                   operations), refinement merges the further pieces above
//                   that it touches; the lane tiles of the block are then
//                   merged along their seams.  Writes the row masks, one
//                   value per piece (block key of its root, or its border
//                   slot), the border record of the block and one global
//                   union-find entry per border component.
//   k_block_merge   step 2, Kernel 2 (Sec. 3.2, Eq. 1-2): only the pixel
//                   pairs that straddle a block edge are examined; the block's
//                   pairs are first joined in a shared-memory union-find and
//                   only the pairs that join two of its sets reach the global
//                   union-find.
//   k_block_write   step 3 (Sec. 3.3): root-find for the block's border slots
//                   in the merged union-find, then expands the per-piece
//                   values over the row masks and writes every label once.
//
// Work items are blocks.  A single image launches one CTA per block; a batch
// of images launches persistent CTAs that take blocks from a device counter
// and find each block's image in a job table (blocks of an image are
// consecutive items, in raster order).
//
// HBM traffic per pixel: 1 B image read, 4 B label write, plus the row masks
// (1/8 B written, 1/8 B read) and 2 B per piece written and read once, most
// of which stay in L2.
#include <algorithm>
#include <cstdint>
#include <deque>
#include <mutex>
#include <vector>

#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "ccl_block.cuh"
#include "ccl_internal.h"

namespace ccl {

__device__ int g_device_error = 0;
// Counters of the coarse-labelling variants (merges, find steps, CAS
// attempts of step 1), accumulated by the counting instantiations only.
__device__ unsigned long long g_variant_ops[3];

// Per-block scratch regions, indexed by the global block (item) index; sized
// for capacity, only the used parts are touched.
struct Scratch {
    uint32_t *masks;   // [blocks][threads][lane tile rows]
    uint4 *vstream;    // [blocks][G::kVChunks][threads]: piece values, 8 per chunk
    uint16_t *edges;   // [blocks][edge entries]
    uint64_t *P;       // [blocks][slots]
    int32_t *nslots;   // [blocks]
};

__device__ __forceinline__ void report(int err) {
    if (err) atomicOr(&g_device_error, err);
}

// Which block the calling CTA works on next.  Thread 0 claims it; the caller
// reads gb (global block) and lb (block inside its image) after the barrier.
struct ItemSlot {
    Job job;
    unsigned gb, lb;
};

__device__ __forceinline__ bool claim_item(const JobTable &jt, int which, unsigned iter, ItemSlot &slot) {
    const unsigned total = jt.hdr ? jt.hdr->total : jt.total;
    if (threadIdx.x == 0) {
        unsigned item;
        if (!jt.hdr) {
            item = iter == 0 ? blockIdx.x : total;
        } else {
            item = atomicAdd(&jt.hdr->counter[which], 1u);
        }
        slot.gb = item;
        if (item < total) {
            if (!jt.hdr) {
                slot.job = jt.single;
                slot.lb = item;
            } else {
                // last job whose first block is <= item
                int lo = 0, hi = (int)jt.hdr->njobs - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (jt.jobs[mid].block0 <= item) lo = mid;
                    else hi = mid - 1;
                }
                slot.job = jt.jobs[lo];
                slot.lb = item - slot.job.block0;
            }
        }
    }
    __syncthreads();
    return slot.gb < total;
}

// ---------------------------------------------------------------------------
// Local root of node x with path halving (stores only ancestors, which a
// concurrent CAS link on a root cannot lose).
__device__ __forceinline__ int local_find(volatile uint16_t *lp, int x, int cap, int &err) {
    for (int i = 0; i < cap; ++i) {
        const int p = lp[x];
        if (p == x) return x;
        const int g = lp[p];
        if (g == p) return p;
        lp[x] = (uint16_t)g;
        x = g;
    }
    err |= kErrGlobalCap;
    return x;
}

// Joins the sets of local nodes a and b, by all 32 lanes of a warp together
// (lanes with valid == false keep step): the larger root is hung under the
// smaller by CAS, and a lane whose CAS failed retries with the new roots.
// True in the lanes whose CAS linked two different sets, so the pairs of
// those lanes form a spanning forest of all the pairs.
__device__ __forceinline__ bool local_union_sync(uint16_t *lp, bool valid, int a, int b, int cap, int &err) {
    volatile uint16_t *vp = lp;
    bool pend = valid, joined = false;
    for (int i = 0; __any_sync(0xFFFFFFFFu, pend); ++i) {
        if (pend) {
            a = local_find(vp, a, cap, err);
            b = local_find(vp, b, cap, err);
            if (a == b || err) {
                pend = false;
            } else {
                if (a < b) { const int t = a; a = b; b = t; }
                if (atomicCAS(reinterpret_cast<unsigned short *>(lp + a), (unsigned short)a, (unsigned short)b) ==
                    (unsigned short)a) {
                    pend = false;
                    joined = true;
                }
            }
        }
        if (i >= cap) {
            if (pend) err |= kErrGlobalCap;
            break;
        }
    }
    return joined;
}

// ---------------------------------------------------------------------------
template <class G, int kCap_>
struct LocalSmem {
    static constexpr int kCap = kCap_;
    static constexpr int kWords = kCap * G::kThreads / 32;  // bitmap words over all entries
    uint16_t par[kCap * G::kThreads];  // list entries, see ccl_block.cuh
    uint32_t mask[G::kLH][G::kThreads];   // row masks
    uint32_t border[kWords];           // bit per entry: root owning a block-border pixel
    uint32_t prefix[kWords];           // border roots in the words before
    uint32_t warp_tot[G::kThreads / 32];
    uint16_t xq[16][G::kThreads];      // further contacts of a band: (piece << 7) | piece above
    uint8_t lastbase[G::kThreads];     // first piece of each lane tile's last band
    int nslots;
    int err;
    ItemSlot item;
};

// Border record entry of a piece value: its slot, or background when the value
// is not a border slot (only possible after an iteration cap was hit).
__device__ __forceinline__ uint16_t border_slot(uint16_t v) {
    return (v & kBorderFlag) ? (uint16_t)(v & 0x7FFF) : kBg;
}

// Block raster key of the smallest pixel of a piece: its first pixel in the
// band's upper row, else (the piece has pixels in the lower row only, where
// it is a row run) its first column.
template <class G>
__device__ __forceinline__ int piece_key(int tx, int ty, int k, uint32_t A, uint32_t rb, int a0) {
    const uint32_t top = A & rb;
    const int row = 2 * k + (top ? 0 : 1);
    const int col = top ? lobit(top) : a0;
    return ((G::kLH * ty + row) << G::kBWLog2) + kLW * tx + col;
}

// 8 two-byte values collected low half first in a 128-bit shift register.
struct HalfQueue {
    uint32_t q0 = 0, q1 = 0, q2 = 0, q3 = 0;
    __device__ __forceinline__ void push(uint32_t v) {
        q0 = __funnelshift_r(q0, q1, 16);
        q1 = __funnelshift_r(q1, q2, 16);
        q2 = __funnelshift_r(q2, q3, 16);
        q3 = (q3 >> 16) | (v << 16);
    }
    __device__ __forceinline__ uint4 bits() const { return make_uint4(q0, q1, q2, q3); }
};

template <class G, bool kConn8, int kMode, bool kCount>
__device__ __forceinline__ void process_local(const Job &job, unsigned lb, unsigned gb, const Scratch &s,
                                              LocalSmem<G, Variant<kConn8, kMode, G::kLH>::kCap> &sm, int cap) {
    using Bd = Bands<kConn8, G::kLH>;
    using V = Variant<kConn8, kMode, G::kLH>;
    constexpr int kCap = V::kCap;
    constexpr int R = Bd::kRows;
    constexpr int NB = Bd::kN;
    constexpr int T = G::kThreads;
    constexpr int kWPT = kCap / 32;  // bitmap words per thread

    const unsigned b = gb;
    const int nbx = job.nbx;
    const int bx = (int)(lb % (unsigned)nbx), by = (int)(lb / (unsigned)nbx);
    const int H = job.H, W = job.W;
    const uint8_t *const img = job.img;
    const size_t pitch = (size_t)job.pitch;
    const bool vec_in = (job.flags & kJobVecIn) != 0;
    const int x0 = bx * G::kBW, y0 = by * G::kBH;
    const int t = threadIdx.x;
    const int tx = t & (G::BLX - 1), ty = t >> G::kBLXLog2;
    const int xl = x0 + kLW * tx, yl = y0 + G::kLH * ty;
    int err = 0;
    unsigned cnt[3] = {0u, 0u, 0u};
    unsigned *const ops = kCount ? cnt : nullptr;

    if (t == 0) sm.err = 0;
    for (int i = t; i < LocalSmem<G, kCap>::kWords; i += T) sm.border[i] = 0u;

    // -- initialization: the lane tile's G::kLH rows as masks (all loads in flight
    // at once; pixels outside the image are background)
    uint32_t mrow[G::kLH];
    if (vec_in && xl + kLW <= W && yl + G::kLH <= H) {
        uint4 raw[2 * G::kLH];
        const uint8_t *p = img + (size_t)yl * pitch + xl;
#pragma unroll
        for (int r = 0; r < G::kLH; ++r) {
            raw[2 * r] = ldg_nc16(p + (size_t)r * pitch);
            raw[2 * r + 1] = ldg_nc16(p + (size_t)r * pitch + 16);
        }
#pragma unroll
        for (int r = 0; r < G::kLH; ++r) mrow[r] = nz16(raw[2 * r]) | (nz16(raw[2 * r + 1]) << 16);
    } else {
#pragma unroll
        for (int r = 0; r < G::kLH; ++r) {
            uint32_t m = 0;
            const int y = yl + r;
            if (y < H && xl < W) {
                const uint8_t *p = img + (size_t)y * pitch + xl;
                const int n = W - xl < kLW ? W - xl : kLW;
                for (int i = 0; i < n; ++i) m |= (uint32_t)(__ldg(p + i) != 0) << i;
            }
            mrow[r] = m;
        }
    }
#pragma unroll
    for (int r = 0; r < G::kLH; ++r) sm.mask[r][t] = mrow[r];

    // -- coarse labelling and refinement, band by band, on the thread's own
    // entries only.  A piece touching the band above takes the first piece it
    // touches there as parent (a root of its own otherwise, keyed by its
    // smallest pixel); every further piece it touches is queued and merged
    // with it once the band is placed.  The 32 lanes of a warp step through
    // their pieces together (lanes past their last piece see a dummy one and
    // store nothing), and the queued merges run as one round per entry.
    uint16_t *const par = sm.par;
    int base_prev = 0, npieces = 0;
    {
        uint32_t pB = 0u, pS = 0u, pE = 0u;  // band above: lower row, piece starts, piece ends
        // queue of a band's further contacts; a full queue (16 entries) is
        // merged by its thread on the spot
        int nq = 0;
        const auto push = [&](int a, int b) {
            if (nq == 16) {
                for (int j = 0; j < 16; ++j) {
                    const int q = sm.xq[j][t];
                    union_private<G, kCap>(par, piece_id<G>(t, q >> 7), piece_id<G>(t, q & 127), cap, err, ops);
                }
                nq = 0;
            }
            sm.xq[nq++][t] = (uint16_t)((a << 7) | b);
        };
#pragma unroll
        for (int k = 0; k < NB; ++k) {
            const uint32_t A = mrow[k * R], Bm = mrow[k * R + R - 1];
            const uint32_t S0 = elem_starts<kConn8, V::kRow>(A, Bm), E0 = elem_ends<kConn8, V::kRow>(A, Bm);
            uint32_t S = S0, E = E0;
            const int nk = __popc(S0);
            const int nmax = __reduce_max_sync(kFull, nk);
            nq = 0;
            for (int i = 0; i < nmax; ++i) {
                const int a0 = lobit(S | 0x80000000u), a1 = lobit(E | 0x80000000u);
                S &= S - 1u;
                E &= E - 1u;
                const bool act = i < nk;
                const uint32_t rb = run_bits(a0, a1);
                const uint32_t P = act ? (pB & touch_range<kConn8>(A & rb)) : 0u;
                // parent: the root the first touched piece above had when it
                // was placed (its entry holds that root's id)
                const int u0 = lobit(P | 0x80000000u);
                const int up = P ? base_prev + __popc(pS & upto(u0)) - 1 : 0;
                const uint16_t ue = par[up * T + t];
                const uint16_t ent = (V::kCol && P) ? ((ue & kRoot) ? (uint16_t)piece_id<G>(t, up) : ue)
                                                    : (uint16_t)(kRoot | piece_key<G>(tx, ty, k, A, rb, a0));
                if (act) par[(npieces + i) * T + t] = ent;
                // (a piece above is a further contact of at most one piece of
                // the band, the leftmost that touches it)
                uint32_t P2 = P ? (V::kCol ? (P & ~upto(piece_end(pE, u0))) : P) : 0u;
                while (P2) {
                    const int u = lobit(P2);
                    push(npieces + i, base_prev + __popc(pS & upto(u)) - 1);
                    P2 &= ~upto(piece_end(pE, u));
                }
            }
            if (!V::kRow) {
                // without coarse labelling along rows, the links between the
                // band's occupied columns are refined like any other contact
                uint32_t L = band_link<kConn8>(A, Bm);
                for (; L; L &= L - 1u) {
                    const int c = lobit(L);
                    const int e = npieces + __popc(S0 & upto(c)) - 1;
                    push(e + 1, e);
                }
            }
            const int nqmax = __reduce_max_sync(kFull, nq);
            for (int j = 0; j < nqmax; ++j) {
                if (j < nq) {
                    const int q = sm.xq[j][t];
                    union_private<G, kCap>(par, piece_id<G>(t, q >> 7), piece_id<G>(t, q & 127), cap, err, ops);
                }
            }
            base_prev = npieces;
            npieces += nk;
            pB = Bm;
            pS = S0;
            pE = E0;
        }
    }
    sm.lastbase[t] = (uint8_t)base_prev;
    __syncthreads();

    // -- block merge of the lane tiles along their seams (Kernel 2's boundary
    // analysis applied inside the block, on the shared lists).  A thread
    // queues the pairs it finds (as the roots their entries name, a pair
    // equal to the one queued before it dropped) and the warp merges the
    // queues in rounds of one pair per lane, whenever a queue may overflow
    // and at the end.
    volatile uint16_t *const vpar = sm.par;
    constexpr int kSQ = 8;  // queue entries per thread, in the space of the band queue
    uint32_t *const sq = reinterpret_cast<uint32_t *>(&sm.xq[0][0]);
    static_assert(sizeof(uint32_t) * kSQ <= sizeof(uint16_t) * 16, "seam queue fits the band queue");
    int nsq = 0;
    uint32_t lastq = 0xFFFFFFFFu;
    const auto seam = [&](bool valid, int a, int b) {
        if (valid) {
            const uint16_t ea = vpar[par_index<G, kCap>(a)], eb = vpar[par_index<G, kCap>(b)];
            const int ra = (ea & kRoot) ? a : (int)ea, rb = (eb & kRoot) ? b : (int)eb;
            const uint32_t q = ((uint32_t)ra << 16) | (uint32_t)rb;
            if (ra != rb && q != lastq) {
                sq[nsq * T + t] = q;
                ++nsq;
                lastq = q;
            }
        }
    };
    const auto flush = [&]() {
        const int m = __reduce_max_sync(kFull, nsq);
        for (int j = 0; j < m; ++j) {
            const bool v = j < nsq;
            const uint32_t q = v ? sq[j * T + t] : 0u;
            union_block_sync<G, kCap>(par, v, (int)(q >> 16), (int)(q & 0xFFFFu), cap, err, ops);
        }
        nsq = 0;
    };
    const auto room = [&](int n) {
        if (__any_sync(kFull, nsq > kSQ - n)) flush();
    };
    {
        const bool hasl = tx > 0;
        const int tl = hasl ? t - 1 : t;
        int mb = 0, lbase = 0;
#pragma unroll
        for (int k = 0; k < NB; ++k) {
            room(3);
            const uint32_t A = mrow[k * R], Bm = mrow[k * R + R - 1];
            const uint32_t lA = sm.mask[k * R][tl], lB = sm.mask[k * R + R - 1][tl];
            const int np = __popc(elem_starts<kConn8, V::kRow>(A, Bm));
            const int lnp = __popc(elem_starts<kConn8, V::kRow>(lA, lB));
            const int me_first = piece_id<G>(t, mb);
            const int l_last = piece_id<G>(tl, lbase + lnp - 1);
            // column 0 of my band k beside column 31 of the left band k
            const uint32_t side = kConn8 ? (A | Bm) & ((lA | lB) >> 31) : (A & (lA >> 31)) | (Bm & (lB >> 31));
            seam(hasl && (side & 1u), me_first, l_last);
            if (kConn8 && k + 1 < NB) {
                const uint32_t nA = mrow[(k + 1) * R];
                const uint32_t lnA = sm.mask[(k + 1) * R][tl];
                const int l_next_last =
                    piece_id<G>(tl, lbase + lnp + __popc(elem_starts<kConn8, V::kRow>(lnA, sm.mask[(k + 1) * R + R - 1][tl])) - 1);
                // lower row of my band k, column 0 ~ upper row of the left band k+1, column 31
                seam(hasl && (Bm & 1u) && (lnA >> 31), me_first, l_next_last);
                // upper row of my band k+1, column 0 ~ lower row of the left band k, column 31
                seam(hasl && (nA & 1u) && (lB >> 31), piece_id<G>(t, mb + np), l_last);
            }
            mb += np;
            lbase += lnp;
        }
    }
    const uint32_t A0 = mrow[0];
    const uint32_t S00 = elem_starts<kConn8, V::kRow>(A0, mrow[R - 1]), E00 = elem_ends<kConn8, V::kRow>(A0, mrow[R - 1]);
    {
        const bool hasu = ty > 0;
        const int tu = hasu ? t - G::BLX : t;
        const uint32_t uA = sm.mask[G::kLH - R][tu], uB = sm.mask[G::kLH - 1][tu];
        const uint32_t uS = elem_starts<kConn8, V::kRow>(uA, uB), uE = elem_ends<kConn8, V::kRow>(uA, uB);
        const int ubase = sm.lastbase[tu];
        uint32_t S = hasu ? S00 : 0u;
        uint32_t E = hasu ? E00 : 0u;
        const int nmax = __reduce_max_sync(kFull, __popc(S));
        for (int i = 0; i < nmax; ++i) {
            const bool act = S != 0u;
            const int a0 = act ? lobit(S) : 0, a1 = act ? lobit(E) : 0;
            S &= S - 1u;
            E &= E - 1u;
            uint32_t P = act ? (uB & touch_range<kConn8>(A0 & run_bits(a0, a1))) : 0u;
            const int me = piece_id<G>(t, i);
            while (__any_sync(kFull, P != 0u)) {
                room(1);
                const bool hp = P != 0u;
                const int u = hp ? lobit(P) : 0;
                seam(hp, me, piece_id<G>(tu, ubase + __popc(uS & upto(u)) - 1));
                if (hp) P &= ~upto(piece_end(uE, u));
            }
        }
        if (kConn8) {
            // corners: the lane tiles up-left and up-right
            room(2);
            const bool ul = hasu && tx > 0 && (A0 & 1u);
            const int tul = ul ? tu - 1 : t;
            const uint32_t ulB = sm.mask[G::kLH - 1][tul];
            seam(ul && (ulB >> 31), piece_id<G>(t, 0),
                 piece_id<G>(tul, sm.lastbase[tul] + __popc(elem_starts<kConn8, V::kRow>(sm.mask[G::kLH - 2][tul], ulB)) - 1));
            const bool ur = hasu && tx + 1 < G::BLX && (A0 >> 31);
            const int tur = ur ? tu + 1 : t;
            seam(ur && (sm.mask[G::kLH - 1][tur] & 1u), piece_id<G>(t, __popc(S00) - 1), piece_id<G>(tur, sm.lastbase[tur]));
        }
        flush();
    }
    __syncthreads();

    // -- compress: every own entry points straight at its root (the finds
    // only read, so every store here is a final root)
    for (int loc = 0; loc < npieces; ++loc) {
        const int id = piece_id<G>(t, loc);
        const int root = find_root_ro<G, kCap>(vpar, id, cap, err);
        if (root != id) vpar[loc * T + t] = (uint16_t)root;
    }
    __syncthreads();

    // -- roots that own a pixel of the block border
    const auto root_of = [&](int id) -> int {
        const uint16_t e = vpar[par_index<G, kCap>(id)];
        return (e & kRoot) ? id : (int)e;
    };
    const auto mark = [&](int id) {
        const int bit = par_index<G, kCap>(root_of(id));
        atomicOr(&sm.border[bit >> 5], 1u << (bit & 31));
    };
    const uint32_t AL = mrow[G::kLH - R], BL = mrow[G::kLH - 1];
    const uint32_t SL = elem_starts<kConn8, V::kRow>(AL, BL), EL = elem_ends<kConn8, V::kRow>(AL, BL);
    if (ty == 0) {
        uint32_t S = S00, E = E00;
        for (int i = 0; S; ++i) {
            const int a0 = lobit(S), a1 = lobit(E);
            S &= S - 1u;
            E &= E - 1u;
            if (A0 & run_bits(a0, a1)) mark(piece_id<G>(t, i));
        }
    }
    if (ty == G::BLY - 1) {
        uint32_t S = SL, E = EL;
        for (int i = base_prev; S; ++i) {
            const int a0 = lobit(S), a1 = lobit(E);
            S &= S - 1u;
            E &= E - 1u;
            if (BL & run_bits(a0, a1)) mark(piece_id<G>(t, i));
        }
    }
    if (tx == 0 || tx == G::BLX - 1) {
        int mb = 0;
#pragma unroll
        for (int k = 0; k < NB; ++k) {
            const uint32_t OR = mrow[k * R] | mrow[k * R + R - 1];
            const int np = __popc(elem_starts<kConn8, V::kRow>(mrow[k * R], mrow[k * R + R - 1]));
            if (tx == 0 && (OR & 1u)) mark(piece_id<G>(t, mb));
            if (tx == G::BLX - 1 && (OR >> 31)) mark(piece_id<G>(t, mb + np - 1));
            mb += np;
        }
    }
    __syncthreads();
    {
        // exclusive popcount prefix over the bitmap: kWPT words per thread,
        // then a scan over threads
        uint32_t c[kWPT], sum = 0;
#pragma unroll
        for (int k = 0; k < kWPT; ++k) {
            c[k] = __popc(sm.border[kWPT * t + k]);
            sum += c[k];
        }
        const int lane = t & 31, w = t >> 5;
        uint32_t incl = sum;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t v = __shfl_up_sync(kFull, incl, d);
            if (lane >= d) incl += v;
        }
        if (lane == 31) sm.warp_tot[w] = incl;
        __syncthreads();
        uint32_t base = 0;
        for (int i = 0; i < w; ++i) base += sm.warp_tot[i];
        uint32_t run = base + incl - sum;
#pragma unroll
        for (int k = 0; k < kWPT; ++k) {
            sm.prefix[kWPT * t + k] = run;
            run += c[k];
        }
        // at most G::kSlots border components exist; more marks only after an
        // iteration cap was hit, and the surplus slots are dropped
        if (t == T - 1) {
            sm.nslots = (int)(base + incl) < G::kSlots ? (int)(base + incl) : G::kSlots;
            if ((int)(base + incl) > G::kSlots) sm.err |= kErrLocalCap;
        }
    }
    __syncthreads();

    // -- one global union-find entry per border component, keyed by its
    // minimum global raster position (ID conversion, Sec. 3.1.4)
    {
        const uint32_t sbase = b * (uint32_t)G::kSlots;
#pragma unroll
        for (int k = 0; k < kWPT; ++k) {
            const int word = kWPT * t + k;
            uint32_t bits = sm.border[word];
            uint32_t slot = sm.prefix[word];
            for (; bits && slot < (uint32_t)G::kSlots; bits &= bits - 1, ++slot) {
                const int at = word * 32 + lobit(bits);
                const int key = vpar[at] & 0x7FFF;
                const uint32_t g = job.key0 + (uint32_t)(y0 + (key >> G::kBWLog2)) * (uint32_t)W +
                                   (uint32_t)(x0 + (key & (G::kBW - 1)));
                s.P[sbase + slot] = pack_slot(g, sbase + slot);
                // from here on the root's entry is its slot (kBorderRoot | slot)
                vpar[at] = (uint16_t)(kBorderRoot | slot);
            }
        }
    }
    __syncthreads();
    // value every piece carries from now on: kBorderFlag | slot of its root,
    // or the block key of its root
    const auto value_of = [&](int id) -> uint16_t {
        uint16_t e = vpar[par_index<G, kCap>(id)];
        if (e < kBorderRoot) e = vpar[par_index<G, kCap>(e)];  // a piece: its entry names the root
        if (e & kRoot) return (uint16_t)(e & 0x7FFF);
        // still a pointer only when an iteration cap cut the merges short
        // (the error word is set then); decode it as block key 0
        if (!(e & kBorderRoot)) return 0;
        return (uint16_t)(kBorderFlag | (e & 0x3FFF));
    };

    // -- border record of the block: the slot of every border pixel, one
    // pixel per thread and step (any thread can read any lane tile's lists)
    uint16_t *const Eb = s.edges + (size_t)b * G::kEdge;
    for (int c = t; c < G::kBW; c += T) {
        // top row: band 0 of the lane tiles with ty == 0
        const int lt = c >> 5, bit = c & 31;
        const uint32_t A = sm.mask[0][lt];
        uint16_t v = kBg;
        if ((A >> bit) & 1u)
            v = border_slot(value_of(piece_id<G>(lt, __popc(elem_starts<kConn8, V::kRow>(A, sm.mask[R - 1][lt]) & upto(bit)) - 1)));
        Eb[G::kEdgeTop + c] = v;
        // bottom row: the last band of the lane tiles with ty == BLY - 1
        const int lb2 = (G::BLY - 1) * G::BLX + lt;
        const uint32_t Bl = sm.mask[G::kLH - 1][lb2];
        v = kBg;
        if ((Bl >> bit) & 1u)
            v = border_slot(value_of(
                piece_id<G>(lb2, sm.lastbase[lb2] + __popc(elem_starts<kConn8, V::kRow>(sm.mask[G::kLH - R][lb2], Bl) & upto(bit)) - 1)));
        Eb[G::kEdgeBottom + c] = v;
    }
    for (int i = t; i < 2 * G::kBH; i += T) {
        // left column (first G::kBH indices) and right column of the block
        const bool right = i >= G::kBH;
        const int r = right ? i - G::kBH : i;
        const int lt = (r / G::kLH) * G::BLX + (right ? G::BLX - 1 : 0);
        const int rr = r & (G::kLH - 1), k = rr / R;
        const uint32_t m = sm.mask[rr][lt];
        uint16_t v = kBg;
        if (right ? (m >> 31) : (m & 1u)) {
            int base = 0;
            for (int j = 0; j < k; ++j) base += __popc(elem_starts<kConn8, V::kRow>(sm.mask[j * R][lt], sm.mask[j * R + R - 1][lt]));
            const int loc = right ? base + __popc(elem_starts<kConn8, V::kRow>(sm.mask[k * R][lt], sm.mask[k * R + R - 1][lt])) - 1
                                  : base;
            v = border_slot(value_of(piece_id<G>(lt, loc)));
        }
        Eb[(right ? G::kEdgeRight : G::kEdgeLeft) + r] = v;
    }
    // -- per-piece values, in piece order
    {
        uint4 *vout = s.vstream + (size_t)b * G::kVChunks * T + t;
        HalfQueue vq;
        for (int loc = 0; loc < npieces; ++loc) {
            vq.push(value_of(piece_id<G>(t, loc)));
            if ((loc & 7) == 7) vout[(size_t)(loc >> 3) * T] = vq.bits();
        }
        if (npieces & 7) {
            for (int k = npieces & 7; k < 8; ++k) vq.push(0);
            vout[(size_t)(npieces >> 3) * T] = vq.bits();
        }
    }
    // -- row masks for the write-out pass
    {
        uint4 *mo = reinterpret_cast<uint4 *>(s.masks + ((size_t)b * T + t) * G::kLH);
#pragma unroll
        for (int q = 0; q < G::kLH / 4; ++q)
            mo[q] = make_uint4(mrow[4 * q], mrow[4 * q + 1], mrow[4 * q + 2], mrow[4 * q + 3]);
    }
    if (err) atomicOr(&sm.err, err);
    if (kCount) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const unsigned v = __reduce_add_sync(kFull, cnt[k]);
            if ((t & 31) == 0 && v) atomicAdd(&g_variant_ops[k], (unsigned long long)v);
        }
    }
    __syncthreads();
    if (t == 0) {
        s.nslots[b] = sm.nslots;
        report(sm.err);
    }
}

template <class G, bool kConn8, int kMode = 0, bool kCount = false>
// (1024 threads per SM, 64 registers; 4-connectivity on 32x8 lane tiles is
// held to 5 CTAs by its shared memory anyway and gets the registers instead)
__global__ void __launch_bounds__(G::kThreads,
                                  (G::kLH == 8 && Variant<kConn8, kMode, G::kLH>::kCap == 128 ? 640 : 1024) /
                                      G::kThreads)
    k_block_local(JobTable jt, Scratch s, int cap) {
    using Sm = LocalSmem<G, Variant<kConn8, kMode, G::kLH>::kCap>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Sm &sm = *reinterpret_cast<Sm *>(smem_raw);
    for (unsigned iter = 0; claim_item(jt, 0, iter, sm.item); ++iter) {
        const Job &job = sm.item.job;
        const unsigned lb = sm.item.lb, gb = sm.item.gb;
        process_local<G, kConn8, kMode, kCount>(job, lb, gb, s, sm, cap);
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Step 2, Kernel 2 (Sec. 3.2, Eq. 1-2): each block examines the pixel pairs
// across its top edge, its left edge and (8-connectivity) its two upper
// corners; the right, bottom and lower corners belong to the neighbouring
// blocks.  A pair that repeats the pair of the neighbouring pixel, or the
// pair the thread linked last, is skipped.  The slots of the block and of the
// blocks above and to the left are joined first in a shared-memory
// union-find (the pairs listed, then joined by whole warps); only the pairs
// that join two of its sets reach the global union-find, all in one round.
template <class G>
struct __align__(16) MergeSmem {  // (16-byte aligned: the edges are staged with 16-byte stores)
    uint16_t up_o[G::kBW], up_p[G::kBW];  // top row of the block, bottom row of the block above
    uint16_t lf_o[G::kBH], lf_p[G::kBH];  // left column of the block, right column of the block to the left
    uint16_t lp[3 * G::kSlots];           // local nodes: own slots, then those above, then those to the left
    uint32_t edge[3 * G::kSlots];         // pairs of local nodes (a << 16) | b: listed, then the joining ones
    int nedge, njoin;
    ItemSlot item;
};

// (kCoherent: the records were written earlier in the same grid, so they are
// read through L2 rather than the non-coherent read-only path)
template <class G, bool kConn8, bool kCoherent = false>
__device__ __forceinline__ void process_merge(const Job &job, unsigned lb, unsigned gb, const Scratch &s,
                                              MergeSmem<G> &sm, int lcap, int gcap, uint32_t bound) {
    constexpr int T = G::kThreads;
    const unsigned b = gb;
    const int nbx = job.nbx;
    const int bx = (int)(lb % (unsigned)nbx), by = (int)(lb / (unsigned)nbx);
    const int t = threadIdx.x;
    const bool up = by > 0, left = bx > 0;
    const unsigned bu = b - (unsigned)nbx, bl = b - 1u;
    const auto ld16 = [](const uint4 *p) { return kCoherent ? __ldcg(p) : __ldg(p); };
    const auto ldn = [&](unsigned blk) { return kCoherent ? __ldcg(s.nslots + blk) : s.nslots[blk]; };
    const int nso = ldn(b);
    const int nsu = up ? ldn(bu) : 0;
    const int nsl = left ? ldn(bl) : 0;
    const uint16_t *Eo = s.edges + (size_t)b * G::kEdge;
    int err = 0;

    // stage the facing edges (16-byte loads) and set up the local union-find
    if (up) {
        const uint4 *src_o = reinterpret_cast<const uint4 *>(Eo + G::kEdgeTop);
        const uint4 *src_p = reinterpret_cast<const uint4 *>(s.edges + (size_t)bu * G::kEdge + G::kEdgeBottom);
        for (int i = t; i < G::kBW / 4; i += T) {
            if (i < G::kBW / 8) reinterpret_cast<uint4 *>(sm.up_o)[i] = ld16(src_o + i);
            else reinterpret_cast<uint4 *>(sm.up_p)[i - G::kBW / 8] = ld16(src_p + (i - G::kBW / 8));
        }
    }
    if (left) {
        const uint4 *src_o = reinterpret_cast<const uint4 *>(Eo + G::kEdgeLeft);
        const uint4 *src_p = reinterpret_cast<const uint4 *>(s.edges + (size_t)bl * G::kEdge + G::kEdgeRight);
        for (int i = t; i < G::kBH / 4; i += T) {
            if (i < G::kBH / 8) reinterpret_cast<uint4 *>(sm.lf_o)[i] = ld16(src_o + i);
            else reinterpret_cast<uint4 *>(sm.lf_p)[i - G::kBH / 8] = ld16(src_p + (i - G::kBH / 8));
        }
    }
    const int nn = nso + nsu + nsl;
    for (int i = t; i < nn; i += T) sm.lp[i] = (uint16_t)i;
    if (t == 0) {
        sm.nedge = 0;
        sm.njoin = 0;
    }
    __syncthreads();

    // at most 3 pairs per top-edge column and per left-edge row
    static_assert(3 * G::kSlots >= 3 * (G::kBW + G::kBH), "the pair list holds every pair of a block");
    static_assert(T % 32 == 0, "the pairs are joined by whole warps");
    uint32_t last = 0xFFFFFFFFu;
    const auto link = [&](int na, int nb) {
        const uint32_t q = ((uint32_t)na << 16) | (uint32_t)nb;
        if (q == last) return;
        last = q;
        const int k = atomicAdd(&sm.nedge, 1);
        if (k < 3 * G::kSlots) sm.edge[k] = q;
    };
    const auto ok = [](uint16_t v, int ns) { return v != kBg && (int)v < ns; };
    if (up) {
        // a run of consecutive columns per thread, so repeats meet the same thread
        constexpr int kPer = (G::kBW + T - 1) / T;
        const int j0 = t * kPer, j1 = j0 + kPer < G::kBW ? j0 + kPer : G::kBW;
        for (int j = j0; j < j1; ++j) {
            const uint16_t a = sm.up_o[j];
            if (!ok(a, nso)) continue;
            const uint16_t aL = j > 0 ? sm.up_o[j - 1] : kBg;
            const uint16_t aR = j + 1 < G::kBW ? sm.up_o[j + 1] : kBg;
            const uint16_t c = sm.up_p[j];
            const uint16_t cL = j > 0 ? sm.up_p[j - 1] : kBg;
            if (ok(c, nsu) && !(aL == a && cL == c)) link(a, nso + c);
            if (kConn8) {
                if (j > 0 && ok(cL, nsu) && aL != a) link(a, nso + cL);
                if (j + 1 < G::kBW) {
                    const uint16_t cR = sm.up_p[j + 1];
                    if (ok(cR, nsu) && aR != a) link(a, nso + cR);
                }
            }
        }
    }
    if (left) {
        for (int j = t; j < G::kBH; j += T) {
            const uint16_t a = sm.lf_o[j];
            if (!ok(a, nso)) continue;
            const uint16_t aU = j > 0 ? sm.lf_o[j - 1] : kBg;
            const uint16_t aD = j + 1 < G::kBH ? sm.lf_o[j + 1] : kBg;
            const uint16_t c = sm.lf_p[j];
            const uint16_t cU = j > 0 ? sm.lf_p[j - 1] : kBg;
            if (ok(c, nsl) && !(aU == a && cU == c)) link(a, nso + nsu + c);
            if (kConn8) {
                if (j > 0 && ok(cU, nsl) && aU != a) link(a, nso + nsu + cU);
                if (j + 1 < G::kBH) {
                    const uint16_t cD = sm.lf_p[j + 1];
                    if (ok(cD, nsl) && aD != a) link(a, nso + nsu + cD);
                }
            }
        }
    }
    __syncthreads();
    // the listed pairs through the shared-memory union-find, a warp-wide step
    // per pair per lane, where the two-step roots of a pair differ; the pairs
    // that join two sets are written back to the front of the list (every
    // index written is below the pairs already read)
    {
        const int nc = sm.nedge < 3 * G::kSlots ? sm.nedge : 3 * G::kSlots;
        volatile uint16_t *vp = sm.lp;
        for (int j0 = 0; j0 < nc; j0 += T) {
            const int j = j0 + t;
            uint32_t q = 0;
            if (j < nc) q = sm.edge[j];
            __syncthreads();
            const int na = (int)(q >> 16), nb = (int)(q & 0xFFFFu);
            const bool need = j < nc && vp[vp[na]] != vp[vp[nb]];
            if (local_union_sync(sm.lp, need, na, nb, lcap, err)) sm.edge[atomicAdd(&sm.njoin, 1)] = q;
            __syncthreads();
        }
    }

    // the joining pairs, then the two corner pairs (8-connectivity)
    const auto slot_of = [&](int node) -> uint32_t {
        if (node < nso) return b * (uint32_t)G::kSlots + (uint32_t)node;
        if (node < nso + nsu) return bu * (uint32_t)G::kSlots + (uint32_t)(node - nso);
        return bl * (uint32_t)G::kSlots + (uint32_t)(node - nso - nsu);
    };
    const int ne = sm.njoin;
    for (int i = t; i < ne; i += T) {
        const uint32_t e = sm.edge[i];
        union_global(s.P, slot_of((int)(e >> 16)), slot_of((int)(e & 0xFFFFu)), gcap, err, bound);
    }
    if (kConn8 && up) {
        if (t == T - 1 && left) {
            const unsigned bd = bu - 1u;
            const uint16_t a = sm.up_o[0], d = kCoherent ? __ldcg(s.edges + (size_t)bd * G::kEdge + G::kEdgeBottom + G::kBW - 1)
                                                         : s.edges[(size_t)bd * G::kEdge + G::kEdgeBottom + G::kBW - 1];
            if (ok(a, nso) && ok(d, ldn(bd)))
                union_global(s.P, b * (uint32_t)G::kSlots + a, bd * (uint32_t)G::kSlots + d, gcap, err, bound);
        }
        if (t == T - 2 && bx + 1 < nbx) {
            const unsigned bd = bu + 1u;
            const uint16_t a = sm.up_o[G::kBW - 1], d = kCoherent ? __ldcg(s.edges + (size_t)bd * G::kEdge + G::kEdgeBottom)
                                                                : s.edges[(size_t)bd * G::kEdge + G::kEdgeBottom];
            if (ok(a, nso) && ok(d, ldn(bd)))
                union_global(s.P, b * (uint32_t)G::kSlots + a, bd * (uint32_t)G::kSlots + d, gcap, err, bound);
        }
    }
    report(err);
}

template <class G, bool kConn8>
__global__ void __launch_bounds__(G::kThreads) k_block_merge(JobTable jt, Scratch s, int lcap, int gcap,
                                                             uint32_t bound) {
    __shared__ MergeSmem<G> sm;
    // launched after step 1, possibly before it has finished (programmatic
    // dependent launch): wait for it, then let the write-out start its
    // prologue while the merge runs
    grid_dependency_wait();
    grid_launch_dependents();
    for (unsigned iter = 0; claim_item(jt, 1, iter, sm.item); ++iter) {
        const Job &job = sm.item.job;
        const unsigned lb = sm.item.lb, gb = sm.item.gb;
        process_merge<G, kConn8>(job, lb, gb, s, sm, lcap, gcap, bound);
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
template <class G>
struct WriteSmem {
    int slot_label[G::kSlots];
    int runlab[G::BLY][G::kBW];          // label of every piece at its start column, one band of all lane tiles
    uint32_t mask[G::kLH][G::kThreads];     // row masks of the block
    ItemSlot item;
};

// Position of (lane tile tx, column c) in a runlab row: the column is XORed
// with tx so that neighbouring lane tiles read by one warp of the copy-out
// spread over the banks.
template <class G>
__device__ __forceinline__ int runlab_index(int tx, int c) { return kLW * tx + (c ^ ((tx & 3) << 3)); }

template <class G, bool kConn8, bool kRow>
__device__ __forceinline__ void process_write(const Job &job, unsigned lb, unsigned gb, const Scratch &s,
                                              WriteSmem<G> &sm, int cap, uint32_t bound) {
    using Bd = Bands<kConn8, G::kLH>;
    constexpr int R = Bd::kRows;
    constexpr int NB = Bd::kN;
    constexpr int T = G::kThreads;

    const unsigned b = gb;
    const int bx = (int)(lb % (unsigned)job.nbx), by = (int)(lb / (unsigned)job.nbx);
    const int H = job.H, W = job.W;
    int32_t *const labels = job.labels;
    const bool vec_out = (job.flags & kJobVecOut) != 0;
    const uint32_t key0 = job.key0;
    const int x0 = bx * G::kBW, y0 = by * G::kBH;
    const int t = threadIdx.x;
    const int tx = t & (G::BLX - 1), ty = t >> G::kBLXLog2;

    // final label of each border slot: root-find in the merged union-find
    // (read-only; every union is complete when this kernel starts)
    const int ns = s.nslots[b];
    int err = 0;
    for (int k = t; k < ns; k += T) {
        uint32_t key;
        find_global_ro(s.P, b * (uint32_t)G::kSlots + (uint32_t)k, key, cap, err, bound);
        sm.slot_label[k] = (int)key + 1;
    }
    report(err);

    const uint4 *mi = reinterpret_cast<const uint4 *>(s.masks + ((size_t)b * T + t) * G::kLH);
    uint32_t mrow[G::kLH];
#pragma unroll
    for (int q = 0; q < G::kLH / 4; ++q) {
        const uint4 m4 = mi[q];
        mrow[4 * q] = m4.x;
        mrow[4 * q + 1] = m4.y;
        mrow[4 * q + 2] = m4.z;
        mrow[4 * q + 3] = m4.w;
    }
#pragma unroll
    for (int r = 0; r < G::kLH; ++r) sm.mask[r][t] = mrow[r];
    // per-piece values, 8 per chunk; the next chunk is always already in flight
    const uint4 *vin = s.vstream + (size_t)b * G::kVChunks * T + t;
    int npieces = 0;
#pragma unroll
    for (int k = 0; k < NB; ++k) {
        npieces += __popc(elem_starts<kConn8, kRow>(mrow[k * R], mrow[k * R + R - 1]));
    }
    const int nchunks = (npieces + 7) >> 3;
    uint4 vq = nchunks > 0 ? vin[0] : make_uint4(0, 0, 0, 0);
    uint4 vnext = nchunks > 1 ? vin[T] : make_uint4(0, 0, 0, 0);
    int vi = 0, vc = 2;
    __syncthreads();

#pragma unroll
    for (int k = 0; k < NB; ++k) {
        // each lane tile: one label per piece of its band k, at the piece start
        uint32_t S = elem_starts<kConn8, kRow>(mrow[k * R], mrow[k * R + R - 1]);
        while (S) {
            const int a0 = lobit(S);
            S &= S - 1u;
            if (vi == 8) {
                vq = vnext;
                if (vc < nchunks) vnext = vin[(size_t)vc * T];
                ++vc;
                vi = 0;
            }
            const uint32_t w = vi < 2 ? vq.x : vi < 4 ? vq.y : vi < 6 ? vq.z : vq.w;
            const uint32_t v = (w >> ((vi & 1) * 16)) & 0xFFFFu;
            ++vi;
            const uint32_t slot = v & 0x7FFFu;
            const int lab = (v & kBorderFlag) ? ((int)slot < ns ? sm.slot_label[slot] : 0)
                                               : (int)(key0 + (uint32_t)(y0 + (int)(v >> G::kBWLog2)) * (uint32_t)W +
                                                       (uint32_t)(x0 + (int)(v & (G::kBW - 1)))) + 1;
            sm.runlab[ty][runlab_index<G>(tx, a0)] = lab;
        }
        __syncthreads();
        // coalesced write-out of the band's rows: every pixel takes the label
        // stored at the start of its piece; a thread covers 4 columns per step
        for (int i = t; i < G::BLY * (G::kBW / 4); i += T) {
            const int ry = i / (G::kBW / 4);
            const int q = i % (G::kBW / 4);         // 4-pixel chunk of the row
            const int ctx = q >> 3;                 // its lane tile
            const int c0 = (q & 7) * 4;             // its first column in the lane tile
            const int x = x0 + 4 * q;
            if (x >= W) continue;
            const uint32_t ma = sm.mask[k * R][ry * G::BLX + ctx];
            const uint32_t mbm = sm.mask[k * R + R - 1][ry * G::BLX + ctx];
            const uint32_t mo = ma | mbm;
            const uint32_t SS = elem_starts<kConn8, kRow>(ma, mbm);
            int lab[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int c = c0 + j;
                lab[j] = ((mo >> c) & 1u) ? sm.runlab[ry][runlab_index<G>(ctx, hibit(SS & upto(c)))] : 0;
            }
#pragma unroll
            for (int rr = 0; rr < R; ++rr) {
                const int y = y0 + G::kLH * ry + k * R + rr;
                if (y >= H) break;
                const uint32_t m = rr == 0 ? ma : mbm;
                int v[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) v[j] = ((m >> (c0 + j)) & 1u) ? lab[j] : 0;
                int32_t *dst = labels + (size_t)y * W + x;
                if (vec_out && x + 4 <= W) {
                    __stcs(reinterpret_cast<int4 *>(dst), make_int4(v[0], v[1], v[2], v[3]));
                } else {
                    __stcs(dst, v[0]);
                    if (x + 1 < W) __stcs(dst + 1, v[1]);
                    if (x + 2 < W) __stcs(dst + 2, v[2]);
                    if (x + 3 < W) __stcs(dst + 3, v[3]);
                }
            }
        }
        __syncthreads();
    }
}

template <class G, bool kConn8, bool kRow = true>
__global__ void __launch_bounds__(G::kThreads) k_block_write(JobTable jt, Scratch s, int cap, uint32_t bound) {
    __shared__ WriteSmem<G> sm;
    for (unsigned iter = 0; claim_item(jt, 2, iter, sm.item); ++iter) {
        const Job &job = sm.item.job;
        const unsigned lb = sm.item.lb, gb = sm.item.gb;
        process_write<G, kConn8, kRow>(job, lb, gb, s, sm, cap, bound);
        __syncthreads();
    }
}

}  // namespace ccl

#include "ccl_pieces.cuh"

// ---------------------------------------------------------------------------
// Host side of this translation unit.

namespace ccl {

namespace {

size_t up256(size_t v) { return (v + 255) & ~(size_t)255; }

struct Layout {
    size_t masks, vstream, edges, P, nslots, total;
};

template <class G>
Layout layout_for(size_t nb) {
    Layout l;
    size_t off = 0;
    l.masks = off;   off += up256(nb * G::kThreads * G::kLH * sizeof(uint32_t));
    l.vstream = off; off += up256(nb * G::kVChunks * G::kThreads * sizeof(uint4));
    l.edges = off;   off += up256(nb * G::kEdge * sizeof(uint16_t));
    l.P = off;       off += up256(nb * G::kSlots * sizeof(uint64_t));
    l.nslots = off;  off += up256(nb * sizeof(int32_t));
    l.total = off;
    return l;
}

template <class G>
Scratch carve(void *ws, size_t nb) {
    const Layout l = layout_for<G>(nb);
    char *p = static_cast<char *>(ws);
    Scratch s;
    s.masks = reinterpret_cast<uint32_t *>(p + l.masks);
    s.vstream = reinterpret_cast<uint4 *>(p + l.vstream);
    s.edges = reinterpret_cast<uint16_t *>(p + l.edges);
    s.P = reinterpret_cast<uint64_t *>(p + l.P);
    s.nslots = reinterpret_cast<int32_t *>(p + l.nslots);
    return s;
}

template <class G>
size_t blocks_of(int H, int W) {
    return (((size_t)W + G::kBW - 1) / G::kBW) * (((size_t)H + G::kBH - 1) / G::kBH);
}

// 512x64, 256x64 and 1024x32 blocks of 32x4 lane tiles, and 512x64 blocks
// of 32x8 lane tiles (fewer, longer per-thread chains: better once an image
// fills every SM many times over)
using G0 = Geo<16, 16, 4>;
using G1 = Geo<8, 16, 4>;
using G2 = Geo<32, 8, 4>;
using G3 = Geo<16, 8, 8>;

// the piece labeller's blocks (8-connectivity): 512 x 64 pixels, 256 threads
using P8 = PGeo<512, 64, 256, true>;
// and for images of few 512 x 64 blocks: 256 x 32 pixels, 128 threads (four
// times the blocks, each a quarter of the work: a shorter chain per block
// while the grid cannot fill the GPU)
using P8s = PGeo<256, 32, 128, true>;
// the same two block shapes under 4-connectivity
using P4 = PGeo<512, 64, 256, false>;
using P4s = PGeo<256, 32, 128, false>;
constexpr size_t kSmallPieceMaxBlocks = 384;  // 512 x 64 blocks (up to about 3500^2 pixels)
static_assert(P8::kBW == G0::kBW && P8::kBH == G0::kBH, "the piece blocks cover the same blocks as 512x64");

template <class PG>
Layout layout_p(size_t nb) {
    Layout l;
    size_t off = 0;
    l.masks = off;   off += up256(nb * PG::kBH * PG::kWords * sizeof(uint32_t));
    l.vstream = off; off += up256(nb * PG::kMaxPieces * sizeof(uint16_t));
    l.edges = off;   off += up256(nb * PG::kEdge * sizeof(uint16_t));
    l.P = off;       off += up256(nb * PG::kSlots * sizeof(uint64_t));
    l.nslots = off;  off += up256(nb * sizeof(int32_t));
    l.total = off;
    return l;
}

template <class PG>
PScratch carve_p(void *ws, size_t nb) {
    const Layout l = layout_p<PG>(nb);
    char *p = static_cast<char *>(ws);
    PScratch s;
    s.masks = reinterpret_cast<uint32_t *>(p + l.masks);
    s.values = reinterpret_cast<uint16_t *>(p + l.vstream);
    s.edges = reinterpret_cast<uint16_t *>(p + l.edges);
    s.P = reinterpret_cast<uint64_t *>(p + l.P);
    s.nslots = reinterpret_cast<int32_t *>(p + l.nslots);
    return s;
}

}  // namespace

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
        if (kind_closes_call(r.kind)) g_timing.pool.push_back(r.b);
    }
}

// Records an event on `s` and, when `kind` >= 0, closes a record for the
// kernel launched since `prev`.  Returns the new event (nullptr when off).
cudaEvent_t timing_mark(cudaStream_t s, cudaEvent_t prev, int kind) {
    std::lock_guard<std::mutex> lk(g_timing.mu);
    if (!g_timing.on) return nullptr;
    // no timing inside stream capture (the events would belong to a graph)
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
        cudaGetLastError();
        return nullptr;
    }
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
    static const char *names[kKernelKinds] = {"k_block_local", "k_block_merge", "k_block_write", "k_piece_local",
                                              "k_piece_write", "k_piece_coop"};
    return (k >= 0 && k < kKernelKinds) ? names[k] : "";
}


namespace {

// Per-device launch facts of one geometry: the block-local kernel needs more
// than the 48 KB of shared memory a launch gets without opting in (the
// opt-in is per device), and persistent grids are sized from occupancy.
struct GeoLaunch {
    bool ready = false;
    int sms = 0;
    int occ_local[2] = {0, 0}, occ_merge[2] = {0, 0}, occ_write[2] = {0, 0};  // [conn8]
};

template <class G, bool kConn8>
bool geo_launch_conn(int dev, GeoLaunch &g) {
    const int bytes = (int)sizeof(LocalSmem<G, Variant<kConn8, 0, G::kLH>::kCap>);
    if (cudaFuncSetAttribute(k_block_local<G, kConn8>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) !=
        cudaSuccess)
        return false;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g.occ_local[kConn8], k_block_local<G, kConn8>,
                                                      G::kThreads, bytes) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g.occ_merge[kConn8], k_block_merge<G, kConn8>,
                                                      G::kThreads, 0) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g.occ_write[kConn8], k_block_write<G, kConn8>,
                                                      G::kThreads, 0) != cudaSuccess)
        return false;
    g.occ_local[kConn8] = std::max(1, g.occ_local[kConn8]);
    g.occ_merge[kConn8] = std::max(1, g.occ_merge[kConn8]);
    g.occ_write[kConn8] = std::max(1, g.occ_write[kConn8]);
    (void)dev;
    return true;
}

template <class G>
bool geo_launch(GeoLaunch &out) {
    static std::mutex mu;
    static GeoLaunch per_dev[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return false;
    std::lock_guard<std::mutex> lk(mu);
    GeoLaunch &g = per_dev[dev];
    if (!g.ready) {
        if (cudaDeviceGetAttribute(&g.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return false;
        if (!geo_launch_conn<G, true>(dev, g) || !geo_launch_conn<G, false>(dev, g)) return false;
        g.ready = true;
    }
    out = g;
    return true;
}

// Default caps: a find walks a strictly decreasing chain, so it cannot take
// more steps than there are list entries (slots); no valid input reaches them.
template <class G>
void caps_for(size_t nb, int cap, int &local_cap, int &global_cap, uint32_t &bound) {
    const long long slots = (long long)nb * G::kSlots;
    local_cap = cap > 0 ? cap : G::kPieceCap * G::kThreads + 16;
    global_cap = cap > 0 ? cap : (int)(slots + 16 < (1LL << 30) ? slots + 16 : (1LL << 30));
    bound = (uint32_t)slots;
}

// The labelling kernel (step 1), the merge (step 2) and the write-out (step
// 3); `phases` selects kPhaseLocalMerge and/or kPhaseWrite.
template <class G>
int launch_table(int conn, const JobTable &jt, unsigned grid_local, unsigned grid_merge, unsigned grid_write,
                 const Scratch &s, int local_cap, int global_cap, uint32_t bound, cudaStream_t stream,
                 int phases = kPhaseLocalMerge | kPhaseWrite) {
    cudaEvent_t ev = timing_mark(stream, nullptr, -1);
    if (conn == 8) {
        if (phases & kPhaseLocalMerge) {
            k_block_local<G, true><<<grid_local, G::kThreads, sizeof(LocalSmem<G, Variant<true, 0, G::kLH>::kCap>),
                                     stream>>>(jt, s, local_cap);
            ev = timing_mark(stream, ev, kKindLocal);
            k_block_merge<G, true><<<grid_merge, G::kThreads, 0, stream>>>(jt, s, local_cap, global_cap, bound);
            ev = timing_mark(stream, ev, kKindMerge);
        }
        if (phases & kPhaseWrite) k_block_write<G, true><<<grid_write, G::kThreads, 0, stream>>>(jt, s, global_cap, bound);
    } else {
        if (phases & kPhaseLocalMerge) {
            k_block_local<G, false><<<grid_local, G::kThreads, sizeof(LocalSmem<G, Variant<false, 0, G::kLH>::kCap>),
                                      stream>>>(jt, s, local_cap);
            ev = timing_mark(stream, ev, kKindLocal);
            k_block_merge<G, false><<<grid_merge, G::kThreads, 0, stream>>>(jt, s, local_cap, global_cap, bound);
            ev = timing_mark(stream, ev, kKindMerge);
        }
        if (phases & kPhaseWrite) k_block_write<G, false><<<grid_write, G::kThreads, 0, stream>>>(jt, s, global_cap, bound);
    }
    if (phases & kPhaseWrite) ev = timing_mark(stream, ev, kKindWrite);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

template <class G>
int launch_single(const uint8_t *img, int H, int W, size_t pitch, int conn, int32_t *labels, void *ws,
                  cudaStream_t stream, int cap, uint32_t key0 = 0, int phases = kPhaseLocalMerge | kPhaseWrite) {
    GeoLaunch gl;
    if (!geo_launch<G>(gl)) return -1;
    JobTable jt{};
    jt.hdr = nullptr;
    jt.jobs = nullptr;
    jt.single.img = img;
    jt.single.labels = labels;
    jt.single.pitch = pitch;
    jt.single.H = H;
    jt.single.W = W;
    jt.single.nbx = (W + G::kBW - 1) / G::kBW;
    jt.single.nby = (H + G::kBH - 1) / G::kBH;
    jt.single.block0 = 0;
    jt.single.key0 = key0;
    jt.single.flags = ((((uintptr_t)img | pitch) & 15) == 0 ? kJobVecIn : 0u) |
                      ((((uintptr_t)labels & 15) == 0 && (W & 3) == 0) ? kJobVecOut : 0u);
    const size_t nb = (size_t)jt.single.nbx * (size_t)jt.single.nby;
    jt.total = (unsigned)nb;
    int local_cap, global_cap;
    uint32_t bound;
    caps_for<G>(nb, cap, local_cap, global_cap, bound);
    return launch_table<G>(conn, jt, (unsigned)nb, (unsigned)nb, (unsigned)nb, carve<G>(ws, nb), local_cap,
                           global_cap, bound, stream, phases);
}

// Launches `kernel` on `stream`; with `pdl` as a programmatic dependent
// launch (it may start before the previous kernel on the stream ends and
// waits for it with griddepcontrol.wait).
template <typename... KArgs, typename... Args>
cudaError_t launch_ex(void (*kernel)(KArgs...), unsigned grid, unsigned block, size_t smem, cudaStream_t stream,
                      bool pdl, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// Per-device set-up of the piece kernels (their shared memory exceeds the 48 KB
// a launch gets without opting in) and their occupancy.
template <class PG>
bool piece_prepare(int &occ_local, int &occ_write, int &sms, int *occ_coop = nullptr, int *occ_merge = nullptr) {
    static std::mutex mu;
    struct Ent {
        bool ready = false;
        int occ_local = 0, occ_write = 0, occ_coop = 0, occ_merge = 0, sms = 0;
    };
    using MG = PGeo<PG::kBW, PG::kBH, (PG::kThreads < 128 ? PG::kThreads : 128), PG::kConn8>;
    static Ent per_dev[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return false;
    std::lock_guard<std::mutex> lk(mu);
    Ent &e = per_dev[dev];
    if (!e.ready) {
        const int bl = (int)sizeof(PLocalSmem<PG>), bw = (int)sizeof(PWriteSmem<PG>);
        if (cudaFuncSetAttribute(k_piece_local<PG>, cudaFuncAttributeMaxDynamicSharedMemorySize, bl) !=
                cudaSuccess ||
            cudaFuncSetAttribute(k_piece_write<PG>, cudaFuncAttributeMaxDynamicSharedMemorySize, bw) !=
                cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&e.occ_local, k_piece_local<PG>, PG::kThreads, bl) !=
                cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&e.occ_write, k_piece_write<PG>, PG::kThreads, bw) !=
                cudaSuccess ||
            cudaFuncSetAttribute(k_piece_coop<PG>, cudaFuncAttributeMaxDynamicSharedMemorySize, bl) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&e.occ_coop, k_piece_coop<PG>, PG::kThreads, bl) !=
                cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&e.occ_merge, k_block_merge<MG, PG::kConn8>, MG::kThreads,
                                                          0) != cudaSuccess ||
            cudaDeviceGetAttribute(&e.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return false;
        e.occ_local = std::max(1, e.occ_local);
        e.occ_write = std::max(1, e.occ_write);
        e.ready = true;
    }
    occ_local = e.occ_local;
    occ_write = e.occ_write;
    sms = e.sms;
    if (occ_coop) *occ_coop = e.occ_coop;
    if (occ_merge) *occ_merge = std::max(1, e.occ_merge);
    return true;
}

// Step 1 (piece labeller), step 2 (the block merge on the border records)
// and step 3 (piece write-out) over the jobs of `jt`.
template <class PG>
int launch_piece_table(const JobTable &jt, unsigned grid_local, unsigned grid_merge, unsigned grid_write,
                       const PScratch &ps, size_t nb, int cap, cudaStream_t stream,
                       int phases = kPhaseLocalMerge | kPhaseWrite, bool chain = false, bool allow_pdl = true) {
    const int local_cap = cap > 0 ? cap : PG::kMaxPieces + 16;
    const long long slots = (long long)nb * PG::kSlots;
    const int global_cap = cap > 0 ? cap : (int)(slots + 16 < (1LL << 30) ? slots + 16 : (1LL << 30));
    const uint32_t bound = (uint32_t)slots;
    Scratch ms{};
    ms.edges = ps.edges;
    ms.P = ps.P;
    ms.nslots = ps.nslots;
    cudaEvent_t ev = timing_mark(stream, nullptr, -1);
    // per-kernel timing records events between the kernels, which a
    // programmatic (overlapping) launch would blur: off while timing
    // (and only between kernels of one call)
    const bool pdl = allow_pdl && ev == nullptr && phases == (kPhaseLocalMerge | kPhaseWrite);
    bool ok = true;
    if (phases & kPhaseLocalMerge) {
        // chained: step 1 may start while the previous call's write-out on
        // this stream still runs (it finishes only after that kernel)
        ok = launch_ex(k_piece_local<PG>, grid_local, PG::kThreads, sizeof(PLocalSmem<PG>), stream,
                       chain && ev == nullptr, jt, ps, local_cap) == cudaSuccess;
        ev = timing_mark(stream, ev, kKindPieceLocal);
        // the merge of many blocks runs on 128 threads per block (more blocks
        // per SM for its latency-bound unions), that of fewer on 256 (a shorter
        // chain per block)
        if (nb >= 1024) {
            using MG = PGeo<PG::kBW, PG::kBH, (PG::kThreads < 128 ? PG::kThreads : 128), PG::kConn8>;
            ok = ok && launch_ex(k_block_merge<MG, PG::kConn8>, grid_merge, MG::kThreads, 0, stream, pdl, jt, ms,
                           local_cap, global_cap, bound) == cudaSuccess;
        } else {
            ok = ok && launch_ex(k_block_merge<PG, PG::kConn8>, grid_merge, PG::kThreads, 0, stream, pdl, jt, ms,
                           local_cap, global_cap, bound) == cudaSuccess;
        }
        ev = timing_mark(stream, ev, kKindMerge);
    }
    if (phases & kPhaseWrite) {
        ok = ok && launch_ex(k_piece_write<PG>, grid_write, PG::kThreads, sizeof(PWriteSmem<PG>), stream, pdl, jt,
                             ps, global_cap, bound) == cudaSuccess;
        ev = timing_mark(stream, ev, kKindPieceWrite);
    }
    return ok && cudaGetLastError() == cudaSuccess ? 0 : -1;
}

template <class PG>
int launch_piece_single(const uint8_t *img, int H, int W, size_t pitch, int32_t *labels, void *ws,
                        cudaStream_t stream, int cap, uint32_t key0 = 0,
                        int phases = kPhaseLocalMerge | kPhaseWrite, bool chain = false) {
    int occ_l = 0, occ_w = 0, sms = 0, occ_c = 0;
    if (!piece_prepare<PG>(occ_l, occ_w, sms, &occ_c)) return -1;
    JobTable jt{};
    jt.single.img = img;
    jt.single.labels = labels;
    jt.single.pitch = pitch;
    jt.single.H = H;
    jt.single.W = W;
    jt.single.nbx = (W + PG::kBW - 1) / PG::kBW;
    jt.single.nby = (H + PG::kBH - 1) / PG::kBH;
    jt.single.block0 = 0;
    jt.single.key0 = key0;
    jt.single.flags = ((((uintptr_t)img | pitch) & 15) == 0 ? kJobVecIn : 0u) |
                      ((((uintptr_t)labels & 15) == 0 && (W & 3) == 0) ? kJobVecOut : 0u);
    const size_t nb = (size_t)jt.single.nbx * (size_t)jt.single.nby;
    jt.total = (unsigned)nb;
    const PScratch ps = carve_p<PG>(ws, nb);
    if (phases == (kPhaseLocalMerge | kPhaseWrite) && nb <= (size_t)occ_c * (size_t)sms) {
        // every block resident at once: the three steps in one cooperative grid
        const int local_cap = cap > 0 ? cap : PG::kMaxPieces + 16;
        const long long slots = (long long)nb * PG::kSlots;
        int global_cap = cap > 0 ? cap : (int)(slots + 16 < (1LL << 30) ? slots + 16 : (1LL << 30));
        uint32_t bound = (uint32_t)slots;
        Scratch ms{};
        ms.edges = ps.edges;
        ms.P = ps.P;
        ms.nslots = ps.nslots;
        PScratch psa = ps;
        int lcap = local_cap;
        void *args[] = {&jt, &psa, &lcap, &ms, &global_cap, &bound};
        cudaEvent_t ev = timing_mark(stream, nullptr, -1);
        const bool ok = cudaLaunchCooperativeKernel((const void *)k_piece_coop<PG>, dim3((unsigned)nb),
                                                    dim3(PG::kThreads), args, sizeof(PLocalSmem<PG>),
                                                    stream) == cudaSuccess;
        timing_mark(stream, ev, kKindPieceCoop);
        return ok && cudaGetLastError() == cudaSuccess ? 0 : -1;
    }
    return launch_piece_table<PG>(jt, (unsigned)nb, (unsigned)nb, (unsigned)nb, ps, nb, cap, stream, phases, chain);
}

template <class G>
int launch_batch(int conn, JobHeader *hdr, const Job *jobs, void *ws, size_t capacity, cudaStream_t stream,
                 int cap) {
    GeoLaunch gl;
    if (!geo_launch<G>(gl)) return -1;
    JobTable jt{};
    jt.hdr = hdr;
    jt.jobs = jobs;
    jt.total = 0;
    int local_cap, global_cap;
    uint32_t bound;
    caps_for<G>(capacity, cap, local_cap, global_cap, bound);
    const int c8 = conn == 8 ? 1 : 0;
    return launch_table<G>(conn, jt, (unsigned)(gl.sms * gl.occ_local[c8]), (unsigned)(gl.sms * gl.occ_merge[c8]),
                           (unsigned)(gl.sms * gl.occ_write[c8]), carve<G>(ws, capacity), local_cap, global_cap,
                           bound, stream);
}

// A batch on the piece labeller: persistent grids (SMs x occupancy) whose
// CTAs claim blocks from the job table's counters.  No programmatic overlap
// between the kernels: a batch is replayed as a captured graph.
template <class PG>
int launch_piece_batch(JobHeader *hdr, const Job *jobs, void *ws, size_t capacity, cudaStream_t stream, int cap) {
    int occ_l = 0, occ_w = 0, sms = 0, occ_m = 0;
    if (!piece_prepare<PG>(occ_l, occ_w, sms, nullptr, &occ_m)) return -1;
    JobTable jt{};
    jt.hdr = hdr;
    jt.jobs = jobs;
    jt.total = 0;
    return launch_piece_table<PG>(jt, (unsigned)(sms * occ_l), (unsigned)(sms * occ_m), (unsigned)(sms * occ_w),
                                  carve_p<PG>(ws, capacity), capacity, cap, stream,
                                  kPhaseLocalMerge | kPhaseWrite, false, false);
}

// One image through a coarse-labelling variant of step 1 (with its
// counters), on 512x64 blocks; steps 2 and 3 as in the method.
template <bool kConn8, int kMode>
int launch_variant_t(const uint8_t *img, int H, int W, size_t pitch, int32_t *labels, void *ws,
                     cudaStream_t stream, int cap) {
    using G = G0;
    using V = Variant<kConn8, kMode, G::kLH>;
    const int bytes = (int)sizeof(LocalSmem<G, V::kCap>);
    if (cudaFuncSetAttribute(k_block_local<G, kConn8, kMode, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             bytes) != cudaSuccess)
        return -1;
    JobTable jt{};
    jt.single.img = img;
    jt.single.labels = labels;
    jt.single.pitch = pitch;
    jt.single.H = H;
    jt.single.W = W;
    jt.single.nbx = (W + G::kBW - 1) / G::kBW;
    jt.single.nby = (H + G::kBH - 1) / G::kBH;
    jt.single.flags = ((((uintptr_t)img | pitch) & 15) == 0 ? kJobVecIn : 0u) |
                      ((((uintptr_t)labels & 15) == 0 && (W & 3) == 0) ? kJobVecOut : 0u);
    const size_t nb = (size_t)jt.single.nbx * (size_t)jt.single.nby;
    jt.total = (unsigned)nb;
    int local_cap, global_cap;
    uint32_t bound;
    caps_for<G>(nb, cap, local_cap, global_cap, bound);
    const Scratch s = carve<G>(ws, nb);
    k_block_local<G, kConn8, kMode, true><<<(unsigned)nb, G::kThreads, bytes, stream>>>(jt, s, local_cap);
    k_block_merge<G, kConn8><<<(unsigned)nb, G::kThreads, 0, stream>>>(jt, s, local_cap, global_cap, bound);
    k_block_write<G, kConn8, V::kRow><<<(unsigned)nb, G::kThreads, 0, stream>>>(jt, s, global_cap, bound);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

template <bool kConn8>
int launch_variant_c(int mode, const uint8_t *img, int H, int W, size_t pitch, int32_t *labels, void *ws,
                     cudaStream_t stream, int cap) {
    switch (mode) {
        case 1: return launch_variant_t<kConn8, 1>(img, H, W, pitch, labels, ws, stream, cap);
        case 2: return launch_variant_t<kConn8, 2>(img, H, W, pitch, labels, ws, stream, cap);
        case 3: return launch_variant_t<kConn8, 3>(img, H, W, pitch, labels, ws, stream, cap);
        default: return launch_variant_t<kConn8, 0>(img, H, W, pitch, labels, ws, stream, cap);
    }
}

}  // namespace

const char *geo_name(int geo) {
    static const char *names[kNumGeo] = {"512x64", "256x64", "1024x32", "512x64x8", "512x64p", "256x32p"};
    return (geo >= 0 && geo < kNumGeo) ? names[geo] : "";
}

void geo_block_shape(int geo, int *bw, int *bh) {
    switch (geo) {
        case 1: *bw = G1::kBW; *bh = G1::kBH; break;
        case 2: *bw = G2::kBW; *bh = G2::kBH; break;
        case 3: *bw = G3::kBW; *bh = G3::kBH; break;
        case 4: *bw = P8::kBW; *bh = P8::kBH; break;
        case 5: *bw = P8s::kBW; *bh = P8s::kBH; break;
        default: *bw = G0::kBW; *bh = G0::kBH; break;
    }
}

size_t geo_blocks(int geo, int H, int W) {
    switch (geo) {
        case 1: return blocks_of<G1>(H, W);
        case 2: return blocks_of<G2>(H, W);
        case 3: return blocks_of<G3>(H, W);
        case 4: return blocks_of<P8>(H, W);
        case 5: return blocks_of<P8s>(H, W);
        default: return blocks_of<G0>(H, W);
    }
}

size_t geo_workspace_bytes(int geo, size_t blocks) {
    switch (geo) {
        case 1: return layout_for<G1>(blocks).total;
        case 2: return layout_for<G2>(blocks).total;
        case 3: return layout_for<G3>(blocks).total;
        case 4: return std::max(layout_p<P8>(blocks).total, layout_p<P4>(blocks).total);
        case 5: return std::max(layout_p<P8s>(blocks).total, layout_p<P4s>(blocks).total);
        default: return layout_for<G0>(blocks).total;
    }
}

// A single image runs on the piece labeller (ccl_pieces.cuh) under either
// connectivity, on 512x64 blocks (256x32 for images of few blocks): its
// pieces span the block width, so a block has no inner seams, and the
// contacts between bands are found for 32 columns at a time by bit
// operations.  The lane-tile kernels above serve batches, the serving loop
// and the coarse-labelling variants.
size_t workspace_bytes(int H, int W) {
    const size_t nb = blocks_of<G0>(H, W);
    const size_t small = blocks_of<G0>(H, W) <= kSmallPieceMaxBlocks
                             ? std::max(layout_p<P8s>(blocks_of<P8s>(H, W)).total,
                                        layout_p<P4s>(blocks_of<P4s>(H, W)).total)
                             : 0;
    return std::max(std::max(std::max(layout_p<P8>(nb).total, layout_p<P4>(nb).total), small),
                    std::max(layout_for<G0>(nb).total, layout_for<G3>(nb).total));
}

int launch_label(const uint8_t *img, int H, int W, size_t pitch, int conn, int32_t *labels, void *ws,
                 cudaStream_t stream, int cap, bool chain) {
    const bool small = blocks_of<G0>(H, W) <= kSmallPieceMaxBlocks;
    constexpr int kAll = kPhaseLocalMerge | kPhaseWrite;
    if (conn == 8)
        return small ? launch_piece_single<P8s>(img, H, W, pitch, labels, ws, stream, cap, 0, kAll, chain)
                     : launch_piece_single<P8>(img, H, W, pitch, labels, ws, stream, cap, 0, kAll, chain);
    return small ? launch_piece_single<P4s>(img, H, W, pitch, labels, ws, stream, cap, 0, kAll, chain)
                 : launch_piece_single<P4>(img, H, W, pitch, labels, ws, stream, cap, 0, kAll, chain);
}

int launch_label_phases(const uint8_t *img, int H, int W, size_t pitch, int conn, uint32_t key0, int32_t *labels,
                        void *ws, cudaStream_t stream, int cap, int phases) {
    if (conn == 8) return launch_piece_single<P8>(img, H, W, pitch, labels, ws, stream, cap, key0, phases);
    return launch_piece_single<P4>(img, H, W, pitch, labels, ws, stream, cap, key0, phases);
}

int label_scratch_view(int H, int W, int conn, void *ws, ScratchView *v) {
    const size_t nb = blocks_of<G0>(H, W);
    char *p = static_cast<char *>(ws);
    const Layout l = conn == 8 ? layout_p<P8>(nb) : layout_p<P4>(nb);
    v->edges = reinterpret_cast<uint16_t *>(p + l.edges);
    v->P = reinterpret_cast<uint64_t *>(p + l.P);
    v->nslots = reinterpret_cast<int32_t *>(p + l.nslots);
    v->nbx = (unsigned)((W + G0::kBW - 1) / G0::kBW);
    v->nby = (unsigned)((H + G0::kBH - 1) / G0::kBH);
    static_assert(P8::kSlots == G0::kSlots && P8::kEdge == G0::kEdge && P8::kEdgeBottom == G0::kEdgeBottom &&
                      P4::kSlots == G0::kSlots && P4::kEdge == G0::kEdge && P4::kEdgeBottom == G0::kEdgeBottom,
                  "the block kinds of strips keep the same border records");
    static_assert(G0::kBW == kStripBW && G0::kBH == kStripBH && G0::kSlots == kStripSlots &&
                      G0::kEdge == kStripEdge && G0::kEdgeBottom == kStripEdgeBottom,
                  "strip constants");
    return 0;
}

int prepare_geo(int geo) {
    GeoLaunch gl;
    int a, b, c;
    switch (geo) {
        case 1: return geo_launch<G1>(gl) ? 0 : -1;
        case 2: return geo_launch<G2>(gl) ? 0 : -1;
        case 3: return geo_launch<G3>(gl) ? 0 : -1;
        case 4: return piece_prepare<P8>(a, b, c) && piece_prepare<P4>(a, b, c) ? 0 : -1;
        case 5: return piece_prepare<P8s>(a, b, c) && piece_prepare<P4s>(a, b, c) ? 0 : -1;
        default: return geo_launch<G0>(gl) ? 0 : -1;
    }
}

int launch_jobs(int geo, int conn, JobHeader *hdr, const Job *jobs, void *ws, size_t capacity,
                cudaStream_t stream, int cap) {
    switch (geo) {
        case 1: return launch_batch<G1>(conn, hdr, jobs, ws, capacity, stream, cap);
        case 2: return launch_batch<G2>(conn, hdr, jobs, ws, capacity, stream, cap);
        case 3: return launch_batch<G3>(conn, hdr, jobs, ws, capacity, stream, cap);
        case 4: return conn == 8 ? launch_piece_batch<P8>(hdr, jobs, ws, capacity, stream, cap)
                                 : launch_piece_batch<P4>(hdr, jobs, ws, capacity, stream, cap);
        case 5: return conn == 8 ? launch_piece_batch<P8s>(hdr, jobs, ws, capacity, stream, cap)
                                 : launch_piece_batch<P4s>(hdr, jobs, ws, capacity, stream, cap);
        default: return launch_batch<G0>(conn, hdr, jobs, ws, capacity, stream, cap);
    }
}

size_t variant_workspace_bytes(int H, int W) { return geo_workspace_bytes(0, geo_blocks(0, H, W)); }

int launch_label_variant(const uint8_t *img, int H, int W, size_t pitch, int conn, int mode, int32_t *labels,
                         void *ws, cudaStream_t stream, int cap) {
    return conn == 8 ? launch_variant_c<true>(mode, img, H, W, pitch, labels, ws, stream, cap)
                     : launch_variant_c<false>(mode, img, H, W, pitch, labels, ws, stream, cap);
}

int variant_counters(unsigned long long *out, bool reset) {
    if (cudaMemcpyFromSymbol(out, g_variant_ops, 3 * sizeof(unsigned long long)) != cudaSuccess) return -1;
    if (reset) {
        const unsigned long long zero[3] = {0, 0, 0};
        if (cudaMemcpyToSymbol(g_variant_ops, zero, sizeof(zero)) != cudaSuccess) return -1;
    }
    return 0;
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
