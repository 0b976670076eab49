// ccl_pieces.cuh -- the block labeller on band pieces indexed across the
// whole block (included once, by ccl_kernels.cu).
//
// A block of kBW x kBH pixels (512 x 64) is cut into bands of two rows.  A
// piece is one connected component of a band: under 8-connectivity a run of
// the OR of the band's two rows, under 4-connectivity a run of columns whose
// neighbours share a row (the two pixels of a column of a band always touch).
// Pieces run across the 32-bit words of a row, so the block has no inner
// seams: Kernel 1's row connection is done by bit operations for the whole
// block width at once.  Every piece gets an index in band order, then column
// order, recomputable from the row masks with a per-band prefix of popcounts.
//
// Step 1 (Kernel 1, Sec. 3.1).  The label-equivalence list of the block has
// one 16-bit entry per piece: kRoot | key for a root (key = block raster
// position of the component's smallest pixel), else the index of its parent.
// Every thread keeps two (band, word) items.  The contact events of each band
// with the band above are found for 32 columns at once by bit operations, one
// event per (piece, piece above) pair.  Column connection: the first event of
// a piece makes the piece above its parent (plain store: no other thread
// writes that entry); a piece without events is a root keyed by its smallest
// pixel.  Refinement: every further event joins its two pieces with a
// warp-synchronous CAS union (links from the larger key to the smaller, Sec.
// 3.1.3), then every entry is compressed to its root.  Roots owning a
// block-border pixel get a border slot and a global union-find entry keyed by
// their minimum global raster position (ID conversion, Sec. 3.1.4).
// Outputs: the row masks, one 16-bit value per piece (border slot or block
// key of its root), the border record and the slot entries.
//
// Step 3 (Sec. 3.3).  The write-out rebuilds the piece index of every column
// from the masks, decodes the piece values into labels in shared memory
// (border slots through a root-find in the merged global union-find) and
// writes every label once, four columns of two rows per thread and step.
#pragma once

namespace ccl {

template <int BW_, int BH_, int T_, bool kConn8_>
struct PGeo {
    static constexpr bool kConn8 = kConn8_;
    static constexpr int kBW = BW_;                      // block width (pixels)
    static constexpr int kBH = BH_;                      // block height
    static constexpr int kThreads = T_;
    static constexpr int kWords = kBW / 32;              // 32-bit words per row
    static constexpr int kWordsLog2 = ilog2(kWords);
    static constexpr int kBands = kBH / 2;
    static constexpr int kBWLog2 = ilog2(kBW);
    static constexpr int kWarps = kThreads / 32;
    static constexpr int kGroup = kBands / kWarps;       // bands placed in order by one warp
    // under 8-connectivity two pieces of a band are at least one empty column
    // apart; under 4-connectivity every column can be a piece of its own
    static constexpr int kBandCap = kConn8 ? kBW / 2 : kBW;
    static constexpr int kMaxPieces = kBands * kBandCap;
    static constexpr int kSlots = kBW + kBH;
    static constexpr int kEdgeTop = 0;
    static constexpr int kEdgeBottom = kBW;
    static constexpr int kEdgeLeft = 2 * kBW;
    static constexpr int kEdgeRight = 2 * kBW + kBH;
    static constexpr int kEdge = 2 * kBW + 2 * kBH;
    // labels decoded per write-out window (a band always fits)
    static constexpr int kLabWindow = 4096 < kMaxPieces / 2 ? 4096 : kMaxPieces / 2;
    static_assert(kBW * kBH <= 32768, "block keys must fit 15 bits");
    static_assert(kMaxPieces <= kBorderRoot, "piece indices must stay below the border-root marker");
    static_assert(kBands <= 32 && kBands % kWarps == 0 && kGroup >= 1, "bands per warp group");
    static_assert((kWords & (kWords - 1)) == 0 && kWords >= 2 && kWords <= 32, "words per row");
    static_assert((kBands * kWords) % kThreads == 0, "band words per thread");
    static_assert(kLabWindow >= kBandCap, "a band fits the label window");
    static_assert((kEdge * 2) % 16 == 0, "border records must stay 16-byte aligned");
};

// Bits lo..hi (inclusive, 0..31) of a word; empty when hi < lo.
__device__ __forceinline__ uint32_t bit_range(int lo, int hi) {
    return hi < lo ? 0u : (upto(hi) & ~((1u << lo) - 1u));
}

// Bits of word w that lie in columns [a, b] of the row.
__device__ __forceinline__ uint32_t word_range(int w, int a, int b) {
    const int lo = a - 32 * w, hi = b - 32 * w;
    if (hi < 0 || lo > 31) return 0u;
    return bit_range(lo < 0 ? 0 : lo, hi > 31 ? 31 : hi);
}

// Per-band tables of a block held as row masks m[kBH][kWords]:
//   S[k][w]  first columns of the band's pieces (a piece continuing from the
//            word before has no start bit here)
//   E[k][w]  last columns of the band's pieces
//   C[k][w]  columns of the lower row of band k-1 that touch the upper row of
//            band k (0 for band 0)
//   pb[k][w] pieces of band k that start in words before w
//   bb[k]    pieces in bands before k (bb[kBands] = all pieces)
// (E and C only when asked for.)  Every thread takes kBands * kWords /
// kThreads (band, word) items; a warp
// holds whole bands, so the word prefix is a segmented warp scan.  The band
// prefix needs the barrier that follows (bb is written by warp 0 after it).
template <class PG, bool kWithEnds, bool kWithContacts>
__device__ __forceinline__ void band_tables(const uint32_t (*m)[PG::kWords], uint32_t (*S)[PG::kWords],
                                            uint32_t (*E)[PG::kWords], uint32_t (*C)[PG::kWords],
                                            uint16_t (*pb)[PG::kWords], uint16_t *bandcnt) {
    constexpr int W = PG::kWords;
    constexpr int kItems = PG::kBands * W / PG::kThreads;
    const int t = threadIdx.x;
#pragma unroll
    for (int j = 0; j < kItems; ++j) {
        const int item = t + j * PG::kThreads;
        const int k = item >> PG::kWordsLog2, w = item & (W - 1);
        const uint32_t A = m[2 * k][w], B = m[2 * k + 1][w];
        const uint32_t Al = w > 0 ? m[2 * k][w - 1] : 0u, Bl = w > 0 ? m[2 * k + 1][w - 1] : 0u;
        const uint32_t Ar = w + 1 < W ? m[2 * k][w + 1] : 0u, Br = w + 1 < W ? m[2 * k + 1][w + 1] : 0u;
        const uint32_t OR = A | B;
        uint32_t s, e;
        if (PG::kConn8) {
            s = OR & ~((OR << 1) | ((Al | Bl) >> 31));
            e = OR & ~((OR >> 1) | ((Ar | Br) << 31));
        } else {
            const uint32_t L = (A & (A >> 1)) | (B & (B >> 1));  // bit c: columns c and c+1 linked
            const uint32_t lin = ((Al >> 31) & A) | ((Bl >> 31) & B);
            const uint32_t lout = ((A >> 31) & Ar & 1u) | ((B >> 31) & Br & 1u);
            s = OR & ~((L << 1) | (lin & 1u));
            e = OR & ~(L | (lout << 31));
        }
        S[k][w] = s;
        if (kWithEnds) E[k][w] = e;
        if (kWithContacts) {
            uint32_t c = 0u;
            if (k > 0) {
                const uint32_t Bu = m[2 * k - 1][w];
                c = PG::kConn8 ? Bu & (A | (A << 1) | (A >> 1) | (Al >> 31) | (Ar << 31)) : Bu & A;
            }
            C[k][w] = c;
        }
        // exclusive prefix of the start counts over the band's words
        const uint32_t cnt = __popc(s);
        uint32_t incl = cnt;
#pragma unroll
        for (int d = 1; d < W; d <<= 1) {
            const uint32_t v = __shfl_up_sync(kFull, incl, d, W);
            if (w >= d) incl += v;
        }
        pb[k][w] = (uint16_t)(incl - cnt);
        if (w == W - 1) bandcnt[k] = (uint16_t)incl;
    }
}

// After the barrier that follows band_tables: warp 0 turns the band counts
// into the band prefix bb[0..kBands].
template <class PG>
__device__ __forceinline__ void band_prefix(const uint16_t *bandcnt, uint16_t *bb) {
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        const uint32_t c = lane < PG::kBands ? bandcnt[lane] : 0u;
        uint32_t incl = c;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t v = __shfl_up_sync(kFull, incl, d);
            if (lane >= d) incl += v;
        }
        if (lane < PG::kBands) bb[lane + 1] = (uint16_t)incl;
        if (lane == 0) bb[0] = 0;
    }
}

// Index of the piece of band k that holds column c (c must be occupied).
template <class PG>
__device__ __forceinline__ int piece_at(const uint32_t (*S)[PG::kWords], const uint16_t (*pb)[PG::kWords],
                                        const uint16_t *bb, int k, int c) {
    const int w = c >> 5;
    return (int)bb[k] + (int)pb[k][w] + __popc(S[k][w] & upto(c & 31)) - 1;
}

// Last column of the piece of band k that holds column c.
template <class PG>
__device__ __forceinline__ int piece_end_at(const uint32_t (*E)[PG::kWords], int k, int c) {
    int w = c >> 5;
    uint32_t e = E[k][w] & ~((1u << (c & 31)) - 1u);
    while (e == 0u && w + 1 < PG::kWords) e = E[k][++w];
    return e ? 32 * w + lobit(e) : PG::kBW - 1;
}

// ---------------------------------------------------------------------------
// Union-find over piece indices (entries as in the header comment).

__device__ __forceinline__ int pfind(volatile uint16_t *par, int x, uint16_t &rentry, int cap, int &err) {
    for (int i = 0; i < cap; ++i) {
        const uint16_t e = par[x];
        if (e & kRoot) { rentry = e; return x; }
        const uint16_t g = par[e];
        if (g & kRoot) { rentry = g; return e; }
        par[x] = g;  // path halving: only non-root entries are rewritten
        x = g;
    }
    err |= kErrLocalCap;
    rentry = kRoot;
    return x;
}

// Root of x with path halving by CAS: a halving store lands only while the
// entry still holds the parent the walk read, so it never overwrites a later
// store of the entry's root.
__device__ __forceinline__ int pfind_cas(uint16_t *par, int x, int cap, int &err) {
    volatile uint16_t *vp = par;
    for (int i = 0; i < cap; ++i) {
        const uint16_t e = vp[x];
        if (e & kRoot) return x;
        const uint16_t g = vp[e];
        if (g & kRoot) return e;
        atomicCAS(reinterpret_cast<unsigned short *>(par + x), (unsigned short)e, (unsigned short)g);
        x = g;
    }
    err |= kErrLocalCap;
    return x;
}

// Merge the lists of a and b, by all 32 lanes of a warp together (lanes with
// valid == false keep step): the root with the larger key is hung under the
// one with the smaller key by CAS; a lane whose CAS failed retries with the
// new roots.
__device__ __forceinline__ void punion_sync(uint16_t *par, bool valid, int a, int b, int cap, int &err) {
    volatile uint16_t *vp = par;
    bool pend = valid;
    for (int i = 0; __any_sync(kFull, pend); ++i) {
        if (pend) {
            uint16_t ea, eb;
            a = pfind(vp, a, ea, cap, err);
            b = pfind(vp, b, eb, cap, err);
            if (a == b || err) {
                pend = false;
            } else {
                if ((ea & 0x7FFF) < (eb & 0x7FFF)) {
                    const int t = a; a = b; b = t;
                    const uint16_t u = ea; ea = eb; eb = u;
                }
                const unsigned short old =
                    atomicCAS(reinterpret_cast<unsigned short *>(par + a), (unsigned short)ea, (unsigned short)b);
                if (old == ea) pend = false;
            }
        }
        if (i >= cap) {
            if (pend) err |= kErrLocalCap;
            break;
        }
    }
}

}  // namespace ccl

namespace ccl {

// Scratch of the piece labeller, per block (indexed by the global block):
// row masks, one value per piece, the border record, the slot entries of the
// global union-find and the slot count.
struct PScratch {
    uint32_t *masks;   // [blocks][kBH][kWords]
    uint16_t *values;  // [blocks][kMaxPieces]
    uint16_t *edges;   // [blocks][kEdge]
    uint64_t *P;       // [blocks][kSlots]
    int32_t *nslots;   // [blocks]
};

// a + b for a row of a band held as kWords 32-bit words, one word per lane of
// a segment of kWords lanes (w = the lane's word): the carries run across the
// words by a Kogge-Stone scan of (generate, propagate).
template <int W>
__device__ __forceinline__ uint32_t row_add(uint32_t a, uint32_t b, int w) {
    const uint32_t s = a + b;
    uint32_t g = s < a ? 1u : 0u;
    uint32_t p = s == 0xFFFFFFFFu ? 1u : 0u;
#pragma unroll
    for (int d = 1; d < W; d <<= 1) {
        const uint32_t g2 = __shfl_up_sync(kFull, g, d, W), p2 = __shfl_up_sync(kFull, p, d, W);
        if (w >= d) {
            g |= p & g2;
            p &= p2;
        }
    }
    const uint32_t cin = __shfl_up_sync(kFull, g, 1, W);
    return s + (w > 0 ? cin : 0u);
}

// Lowest bit of every run of R that holds a bit of M (M a subset of R), for a
// row of a band spread over a segment of lanes: the add clears each run from
// its lowest seed upwards except the higher seeds, so the lowest seed is the
// only bit of M left in (R + M) ^ R.
template <int W>
__device__ __forceinline__ uint32_t lowest_per_run(uint32_t R, uint32_t M, int w) {
    return M & (row_add<W>(R, M, w) ^ R);
}

// Segments: the runs of R, each also cut before every bit of Bs (a segment
// may start inside a run).  Lowest bit of M (a subset of R) in every segment:
// a seed on a segment's first column is the lowest of its segment; otherwise
// the lowest seed of the segment's tail (R without the first columns), whose
// run starts one column later, unless that tail follows a seeded first
// column.
template <int W>
__device__ __forceinline__ uint32_t lowest_per_seg(uint32_t R, uint32_t Bs, uint32_t M, int w) {
    const uint32_t R2 = R & ~Bs;
    const uint32_t mb = M & Bs;
    const uint32_t prev = __shfl_up_sync(kFull, mb, 1, W);
    const uint32_t after = ((mb << 1) | (w > 0 ? prev >> 31 : 0u)) & R2;
    const uint32_t T = R2 & ~row_add<W>(R2, after, w);
    return mb | (lowest_per_run<W>(R2, M & R2, w) & ~T);
}

// Bits of every segment (as above) from its seed to its last column, for at
// most one seed M1 per segment.
template <int W>
__device__ __forceinline__ uint32_t fill_per_seg(uint32_t R, uint32_t Bs, uint32_t M1, int w) {
    const uint32_t R2 = R & ~Bs;
    const uint32_t mb = M1 & Bs;
    const uint32_t prev = __shfl_up_sync(kFull, mb, 1, W);
    const uint32_t seeds = (M1 & R2) | (((mb << 1) | (w > 0 ? prev >> 31 : 0u)) & R2);
    return mb | (R2 & ~row_add<W>(R2, seeds, w));
}

template <class PG>
struct PLocalSmem {
    static constexpr int kCandCap = 2048;  // union candidates per pass
    uint32_t m[PG::kBH][PG::kWords];      // row masks
    uint32_t S[PG::kBands][PG::kWords];   // piece starts
    uint16_t pb[PG::kBands][PG::kWords];  // pieces of the band in earlier words
    uint16_t bandcnt[PG::kBands];
    uint16_t bb[PG::kBands + 1];          // pieces in earlier bands
    alignas(16) uint32_t cand[kCandCap];  // union candidates: piece << 16 | piece above
    uint16_t par[PG::kMaxPieces];         // label-equivalence list entries
    uint32_t border[PG::kMaxPieces / 32]; // bit per entry: root owning a block-border pixel
    uint32_t prefix[PG::kMaxPieces / 32]; // border roots in the words before
    uint32_t warp_tot[PG::kWarps];
    int nslots;
    int err;
    ItemSlot item;
};

// Piece starts (first columns) and piece ends (last columns) of a band under
// 4-connectivity, from its rows A, B and the bits of the neighbouring words:
// columns c and c+1 are one piece when they share a row.
__device__ __forceinline__ uint32_t starts4(uint32_t A, uint32_t B, uint32_t Al, uint32_t Bl) {
    const uint32_t L = (A & (A >> 1)) | (B & (B >> 1));
    const uint32_t lin = ((Al >> 31) & A) | ((Bl >> 31) & B);
    return (A | B) & ~((L << 1) | (lin & 1u));
}
__device__ __forceinline__ uint32_t ends4(uint32_t A, uint32_t B, uint32_t Ar, uint32_t Br) {
    const uint32_t L = (A & (A >> 1)) | (B & (B >> 1));
    const uint32_t lout = ((A >> 31) & Ar & 1u) | ((B >> 31) & Br & 1u);
    return (A | B) & ~(L | (lout << 31));
}

// Contact events of band k with band k-1 under 4-connectivity: a pixel A[c]
// of the upper row of band k touches the band above only at Bu[c], so the
// contacts are E = A & Bu.  A piece P of band k and a piece U of band k-1
// are both intervals of columns, and a run of E lies in one (P, U) pair (two
// neighbouring columns of A, or of Bu, are one piece); the pairs are the
// segments of R = OR & ORu cut at the starts of the pieces of either band.
// D1 keeps the lowest contact of every segment (one event per pair), FE the
// lowest D1 of every piece, TA the first upper-row pixel of every piece, RE
// the last column of every piece without events (the outputs of
// band_events; no L or R events exist).
template <class PG, int kItems>
__device__ __forceinline__ void band_events4(const PLocalSmem<PG> &sm, uint32_t (&D1)[kItems],
                                             uint32_t (&EL)[kItems], uint32_t (&ER)[kItems],
                                             uint32_t (&FE)[kItems], uint32_t (&TA)[kItems],
                                             uint32_t (&RE)[kItems]) {
    constexpr int W = PG::kWords;
#pragma unroll
    for (int j = 0; j < kItems; ++j) {
        const int item = threadIdx.x + j * PG::kThreads;
        const int k = item >> PG::kWordsLog2, w = item & (W - 1);
        const uint32_t A = sm.m[2 * k][w], B = sm.m[2 * k + 1][w], OR = A | B;
        const uint32_t Al = w > 0 ? sm.m[2 * k][w - 1] : 0u, Bl = w > 0 ? sm.m[2 * k + 1][w - 1] : 0u;
        const uint32_t Ar = w + 1 < W ? sm.m[2 * k][w + 1] : 0u, Br = w + 1 < W ? sm.m[2 * k + 1][w + 1] : 0u;
        const uint32_t Sk = starts4(A, B, Al, Bl);
        uint32_t Au = 0u, Bu = 0u, Sku = 0u;
        if (k > 0) {
            Au = sm.m[2 * k - 2][w];
            Bu = sm.m[2 * k - 1][w];
            const uint32_t Aul = w > 0 ? sm.m[2 * k - 2][w - 1] : 0u, Bul = w > 0 ? sm.m[2 * k - 1][w - 1] : 0u;
            Sku = starts4(Au, Bu, Aul, Bul);
        }
        const uint32_t R = OR & (Au | Bu);
        D1[j] = lowest_per_seg<W>(R, (Sk | Sku) & R, A & Bu, w);
        EL[j] = 0u;
        ER[j] = 0u;
        FE[j] = lowest_per_seg<W>(OR, Sk, D1[j], w);
        TA[j] = lowest_per_seg<W>(OR, Sk, A, w);
        RE[j] = ends4(A, B, Ar, Br) & ~fill_per_seg<W>(OR, Sk, FE[j], w);
    }
}

// Contact events of band k with band k-1 under 8-connectivity, for the
// (band, word) items of the calling thread (a warp holds whole bands).  A
// pixel A[c] of the upper row of band k touches the lower row Bu of band k-1
// at c-1, c or c+1.  If band k-1 occupies column c, every such touch is with
// the piece of band k-1 that holds c: an E1 event at c.  Otherwise the
// touches at c-1 and c+1 are with two different pieces: L and R events at c.
// Every E1 event of one run of (OR & ORu) joins the same two pieces, so D1
// keeps the lowest E1 event of each such run.  An L event at c whose column
// c-1 holds an E1 event joins the same two pieces as that E1 event (c-1 and c
// lie in one run of band k, c-1 in the run of band k-1 the L event names), so
// it is dropped; likewise an R event next to an E1 event at c+1.
//
// A piece P of band k and a piece U of band k-1 meet in at most one run of
// (OR & ORu) (the overlap of two intervals), and an R event names U only at
// the column before U's first column, an L event only after its last.  So one
// event per (P, U) pair remains when (a) the D1 event of a run is dropped if
// an R event seeds the run's first column, and (b) an L event is dropped if
// the run of (OR & ORu) ending next to it holds a kept D1 or R seed (the fill
// R & ~(R + seed) marks a run from its seed to its last column).
//
// FE is the first event of every piece of band k (lowest bit of D1 | EL | ER
// per run of its OR), TA the first upper-row pixel of every piece (its
// smallest pixel, when it has one) and RE the last column of every piece
// without events.  Each thread keeps the masks of its items in registers:
// every later pass over (band, word) items uses the same items.
template <class PG, int kItems>
__device__ __forceinline__ void band_events(const PLocalSmem<PG> &sm, uint32_t (&D1)[kItems], uint32_t (&EL)[kItems],
                                            uint32_t (&ER)[kItems], uint32_t (&FE)[kItems], uint32_t (&TA)[kItems],
                                            uint32_t (&RE)[kItems]) {
    constexpr int W = PG::kWords;
    if constexpr (!PG::kConn8) {
        band_events4<PG, kItems>(sm, D1, EL, ER, FE, TA, RE);
    } else {
#pragma unroll
        for (int j = 0; j < kItems; ++j) {
            const int item = threadIdx.x + j * PG::kThreads;
            const int k = item >> PG::kWordsLog2, w = item & (W - 1);
            const int ku = k > 0 ? k - 1 : 0;
            const uint32_t A = sm.m[2 * k][w], B = sm.m[2 * k + 1][w], OR = A | B;
            const uint32_t Bu = k > 0 ? sm.m[2 * ku + 1][w] : 0u;
            const uint32_t ORu = k > 0 ? (sm.m[2 * ku][w] | Bu) : 0u;
            const uint32_t Bul = (k > 0 && w > 0) ? sm.m[2 * ku + 1][w - 1] : 0u;
            const uint32_t Bur = (k > 0 && w + 1 < W) ? sm.m[2 * ku + 1][w + 1] : 0u;
            const uint32_t BuL = (Bu << 1) | (Bul >> 31);  // bit c: Bu[c-1]
            const uint32_t BuR = (Bu >> 1) | (Bur << 31);  // bit c: Bu[c+1]
            const uint32_t E1 = A & ORu & (Bu | BuL | BuR);
            // E1 of the neighbouring columns (bits from the neighbouring words)
            const uint32_t Al = w > 0 ? sm.m[2 * k][w - 1] : 0u, Ar = w + 1 < W ? sm.m[2 * k][w + 1] : 0u;
            const uint32_t ORur = (k > 0 && w + 1 < W) ? (sm.m[2 * ku][w + 1] | Bur) : 0u;
            // E1 at column 32w-1 under an L event at 32w (Bu there is set): A there
            const uint32_t e1l = (Al >> 31) & (Bul >> 31) & 1u;
            // E1 at column 32w+32 under an R event at 32w+31 (Bu there is set)
            const uint32_t e1r = Ar & ORur & 1u & (((Bur & 1u) | (Bu >> 31) | ((Bur >> 1) & 1u)) ? 1u : 0u);
            const uint32_t E1l = (E1 << 1) | e1l;         // bit c: E1[c-1]
            const uint32_t E1r = (E1 >> 1) | (e1r << 31); // bit c: E1[c+1]
            const uint32_t el0 = A & ~ORu & BuL & ~E1l;
            ER[j] = A & ~ORu & BuR & ~E1r;
            const uint32_t R = OR & ORu;
            const uint32_t d1 = lowest_per_run<W>(R, E1, w);
            // runs of R whose first column follows an R event: (a)
            const uint32_t erp = __shfl_up_sync(kFull, ER[j], 1, W);
            const uint32_t ers = ((ER[j] << 1) | (w > 0 ? erp >> 31 : 0u)) & R;
            const uint32_t G = R & ~row_add<W>(R, ers, w);
            D1[j] = d1 & ~G;
            // runs of R holding a kept seed, from the seed on: (b)
            const uint32_t F2 = R & ~row_add<W>(R, D1[j] | ers, w);
            const uint32_t f2p = __shfl_up_sync(kFull, F2, 1, W);
            EL[j] = el0 & ~((F2 << 1) | (w > 0 ? f2p >> 31 : 0u));
            FE[j] = lowest_per_run<W>(OR, D1[j] | EL[j] | ER[j], w);
            TA[j] = lowest_per_run<W>(OR, A, w);
            // last columns of the runs without an event
            const uint32_t orn = __shfl_down_sync(kFull, OR, 1, W);
            const uint32_t endm = OR & ~((OR >> 1) | ((w + 1 < W ? orn : 0u) << 31));
            RE[j] = endm & row_add<W>(OR, FE[j], w);
        }
    }
}

// Block raster key of the smallest pixel of piece [a0, a1] of band k: its
// first pixel in the band's upper row, else its first column (a piece with
// no upper-row pixel starts with a lower-row pixel).
template <class PG>
__device__ __forceinline__ int pkey(const uint32_t (*m)[PG::kWords], int k, int a0, int a1) {
    for (int w = a0 >> 5; w <= (a1 >> 5); ++w) {
        const uint32_t top = m[2 * k][w] & word_range(w, a0, a1);
        if (top) return ((2 * k) << PG::kBWLog2) + 32 * w + lobit(top);
    }
    return ((2 * k + 1) << PG::kBWLog2) + a0;
}

// Root of x as its entry names it (one step; exact while entries point at
// roots, an ancestor otherwise).
__device__ __forceinline__ int proot1(const volatile uint16_t *par, int x) {
    const uint16_t e = par[x];
    return (e & kRoot) ? x : (int)e;
}

// Root of x within two steps (an ancestor when the chain is longer).
__device__ __forceinline__ int proot2(const volatile uint16_t *par, int x) {
    const uint16_t e = par[x];
    if (e & kRoot) return x;
    const uint16_t g = par[e];
    return (g & kRoot) ? (int)e : (int)g;
}

// Value every piece carries to the write-out: kBorderFlag | slot of its root,
// or the block key of its root (entries compressed: a piece's entry is its
// root's index or the root's own entry).
__device__ __forceinline__ uint16_t pvalue(const volatile uint16_t *par, int i) {
    uint16_t e = par[i];
    if (e < kBorderRoot) e = par[e];
    if (e & kRoot) return (uint16_t)(e & 0x7FFF);
    if (!(e & kBorderRoot)) return 0;  // only after an iteration cap cut the merges short
    return (uint16_t)(kBorderFlag | (e & 0x3FFF));
}

// Row and column (block coordinates) of border item j: top row, bottom row,
// left column, right column, in the order of the border record.
template <class PG>
__device__ __forceinline__ void border_pos(int j, int &row, int &col) {
    if (j < PG::kEdgeBottom) { row = 0; col = j; }
    else if (j < PG::kEdgeLeft) { row = PG::kBH - 1; col = j - PG::kEdgeBottom; }
    else if (j < PG::kEdgeRight) { row = j - PG::kEdgeLeft; col = 0; }
    else { row = j - PG::kEdgeRight; col = PG::kBW - 1; }
}

// Upper-band column of event bit c (a column of band k) of class d1 / el /
// er: the column of band k-1 whose piece the event joins.
__device__ __forceinline__ int event_upper_col(int col, bool d1, bool el) {
    return d1 ? col : (el ? col - 1 : col + 1);
}

template <class PG>
__device__ __forceinline__ void process_plocal(const Job &job, unsigned lb, unsigned gb, const PScratch &s,
                                               PLocalSmem<PG> &sm, int cap) {
    constexpr int W = PG::kWords;
    constexpr int T = PG::kThreads;
    constexpr int kBorderWords = PG::kMaxPieces / 32;
    constexpr int kItems = PG::kBands * W / T;
    const unsigned b = gb;
    const int nbx = job.nbx;
    const int bx = (int)(lb % (unsigned)nbx), by = (int)(lb / (unsigned)nbx);
    const int H = job.H, Wd = job.W;
    const uint8_t *const img = job.img;
    const size_t pitch = (size_t)job.pitch;
    const int x0 = bx * PG::kBW, y0 = by * PG::kBH;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    int err = 0;

    if (t == 0) sm.err = 0;
    for (int i = t; i < kBorderWords; i += T) sm.border[i] = 0u;

    // -- the block as row masks: every (row, word) item is 32 bytes of image;
    // all loads of a thread are in flight at once when the block lies inside
    // the image, pixels outside the image are background
    {
        constexpr int kLoads = PG::kBH * W / T;
        const bool inside = (job.flags & kJobVecIn) && x0 + PG::kBW <= Wd && y0 + PG::kBH <= H;
        if (inside) {
            uint4 raw[2 * kLoads];
#pragma unroll
            for (int j = 0; j < kLoads; ++j) {
                const int item = t + j * T;
                const int r = item >> PG::kWordsLog2, w = item & (W - 1);
                const uint8_t *p = img + (size_t)(y0 + r) * pitch + x0 + 32 * w;
                raw[2 * j] = ldg_nc16(p);
                raw[2 * j + 1] = ldg_nc16(p + 16);
            }
#pragma unroll
            for (int j = 0; j < kLoads; ++j) {
                const int item = t + j * T;
                sm.m[item >> PG::kWordsLog2][item & (W - 1)] = nz16(raw[2 * j]) | (nz16(raw[2 * j + 1]) << 16);
            }
        } else {
            for (int item = t; item < PG::kBH * W; item += T) {
                const int r = item >> PG::kWordsLog2, w = item & (W - 1);
                const int y = y0 + r, x = x0 + 32 * w;
                uint32_t mk = 0;
                if (y < H && x < Wd) {
                    const uint8_t *p = img + (size_t)y * pitch + x;
                    const int n = Wd - x < 32 ? Wd - x : 32;
                    for (int i = 0; i < n; ++i) mk |= (uint32_t)(__ldg(p + i) != 0) << i;
                }
                sm.m[r][w] = mk;
            }
        }
    }
    __syncthreads();
    // -- row connection (the pieces, by bit operations) and the contact
    // events of every band with the band above
    band_tables<PG, false, false>(sm.m, sm.S, nullptr, nullptr, sm.pb, sm.bandcnt);
    uint32_t evD1[kItems], evEL[kItems], evER[kItems], evFE[kItems], evTA[kItems], evRE[kItems];
    band_events<PG, kItems>(sm, evD1, evEL, evER, evFE, evTA, evRE);
    __syncthreads();
    band_prefix<PG>(sm.bandcnt, sm.bb);
    __syncthreads();
    const int n = sm.bb[PG::kBands];
    volatile uint16_t *const vpar = sm.par;
    uint16_t *const par = sm.par;
    int qbase[kItems], ubase[kItems];
    uint32_t Sw[kItems], Suw[kItems];
#pragma unroll
    for (int j = 0; j < kItems; ++j) {
        const int item = t + j * T;
        const int k = item >> PG::kWordsLog2, w = item & (W - 1);
        qbase[j] = (int)sm.bb[k] + (int)sm.pb[k][w] - 1;
        Sw[j] = sm.S[k][w];
        ubase[j] = k > 0 ? (int)sm.bb[k - 1] + (int)sm.pb[k - 1][w] - 1 : 0;
        Suw[j] = k > 0 ? sm.S[k - 1][w] : 0u;
    }
    // index of the piece above that event bit c (class d1 / el / er) joins
    const auto upper_piece = [&](int j, int k, int w, int c, bool d1, bool el) -> int {
        const int uc = event_upper_col(32 * w + c, d1, el);
        if ((uc >> 5) == w) return ubase[j] + __popc(Suw[j] & upto(uc & 31));
        return piece_at<PG>(sm.S, sm.pb, sm.bb, k - 1, uc);
    };
    // -- one entry per piece.  Column connection (coarse labelling): the first
    // event of a piece names the piece above that becomes its parent (a
    // smaller key, so the entries form a forest).  A piece without events is
    // a root keyed by its smallest pixel: its first upper-row pixel, else the
    // first column of its lower row.
#pragma unroll
    for (int j = 0; j < kItems; ++j) {
        const int item = t + j * T;
        const int k = item >> PG::kWordsLog2, w = item & (W - 1);
        const uint32_t d1 = evD1[j], el = evEL[j];
        for (uint32_t fe = evFE[j]; fe; fe &= fe - 1u) {
            const int c = lobit(fe);
            const int q = qbase[j] + __popc(Sw[j] & upto(c));
            vpar[q] = (uint16_t)upper_piece(j, k, w, c, (d1 >> c) & 1u, (el >> c) & 1u);
        }
        for (uint32_t re = evRE[j]; re; re &= re - 1u) {
            const int c = lobit(re);
            const int q = qbase[j] + __popc(Sw[j] & upto(c));
            const uint32_t sb = Sw[j] & upto(c);
            int key;
            if (sb) {
                const int s0 = 31 - __clz(sb);
                const uint32_t tab = evTA[j] & upto(c) & ~((1u << s0) - 1u);
                key = tab ? (((2 * k) << PG::kBWLog2) + 32 * w + lobit(tab))
                          : (((2 * k + 1) << PG::kBWLog2) + 32 * w + s0);
            } else {
                // the run began in an earlier word: its first column is the
                // last start of the nearest earlier word that holds one
                int a0 = 0;
                for (int w2 = w - 1; w2 >= 0; --w2) {
                    const uint32_t s2 = sm.S[k][w2];
                    if (s2) {
                        a0 = 32 * w2 + 31 - __clz(s2);
                        break;
                    }
                }
                key = pkey<PG>(sm.m, k, a0, 32 * w + c);
            }
            vpar[q] = (uint16_t)(kRoot | key);
        }
    }
    __syncthreads();
    // -- one round of pointer jumping: every link to its grandparent (an
    // ancestor either way when another thread's store races with the read),
    // halving the coarse links' chains before the unions walk them
    for (int i = t; i < n; i += T) {
        const uint16_t e = vpar[i];
        if (!(e & kRoot)) {
            const uint16_t g = vpar[e];
            if (!(g & kRoot)) vpar[i] = g;
        }
    }
    __syncthreads();
    // -- refinement: every other event joins its two pieces; the CAS union
    // runs only where the roots their entries name differ (the finds of the
    // unions halve the paths of the coarse links as they go).  The events are
    // first packed into a list of (piece, piece above) pairs, so that every
    // lane takes one per step.
    {
        constexpr int kCand = PLocalSmem<PG>::kCandCap;
        uint32_t *const cand = sm.cand;
        uint32_t cnt[kItems], sum = 0;
#pragma unroll
        for (int j = 0; j < kItems; ++j) {
            const uint32_t fe = evFE[j], el = evEL[j];
            cnt[j] = __popc(evD1[j] & ~fe) + __popc(el & ~fe) + __popc(evER[j] & ~(fe & ~el));
            sum += cnt[j];
        }
        uint32_t incl = sum;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t v = __shfl_up_sync(kFull, incl, d);
            if (lane >= d) incl += v;
        }
        if (lane == 31) sm.warp_tot[warp] = incl;
        __syncthreads();
        uint32_t base = 0, total = 0;
        for (int q = 0; q < PG::kWarps; ++q) {
            if (q < warp) base += sm.warp_tot[q];
            total += sm.warp_tot[q];
        }
        base += incl - sum;
        for (uint32_t lo = 0; lo < total; lo += kCand) {
            const uint32_t hi = lo + kCand;
            uint32_t at = base;
#pragma unroll
            for (int j = 0; j < kItems; ++j) {
                const int item = t + j * T;
                const int k = item >> PG::kWordsLog2, w = item & (W - 1);
                if (at + cnt[j] > lo && at < hi) {
                    const uint32_t fe = evFE[j], el = evEL[j];
                    uint32_t ud = evD1[j] & ~fe, ul = el & ~fe, ur = evER[j] & ~(fe & ~el);
                    uint32_t idx = at;
                    for (; (ud | ul | ur) && idx < hi; ++idx) {
                        int c;
                        bool isd = false, isl = false;
                        if (ud) { c = lobit(ud); ud &= ud - 1u; isd = true; }
                        else if (ul) { c = lobit(ul); ul &= ul - 1u; isl = true; }
                        else { c = lobit(ur); ur &= ur - 1u; }
                        if (idx < lo) continue;
                        const int q = qbase[j] + __popc(Sw[j] & upto(c));
                        cand[idx - lo] = ((uint32_t)q << 16) | (uint32_t)upper_piece(j, k, w, c, isd, isl);
                    }
                }
                at += cnt[j];
            }
            __syncthreads();
            const uint32_t nc = total - lo < (uint32_t)kCand ? total - lo : (uint32_t)kCand;
            for (uint32_t j0 = 0; j0 < nc; j0 += T) {
                const uint32_t j = j0 + t;
                int q = 0, iu = 0;
                bool need = false;
                if (j < nc) {
                    const uint32_t e = cand[j];
                    q = (int)(e >> 16);
                    iu = (int)(e & 0xFFFFu);
                    need = proot2(vpar, q) != proot2(vpar, iu);
                }
                punion_sync(par, need, q, iu, cap, err);
            }
            __syncthreads();
        }
    }
    // -- compress: every entry points straight at its root (each entry's
    // final store is made by its own thread; the halving stores of the
    // other walks are CAS and cannot undo it)
    for (int i = t; i < n; i += T) {
        const int r = pfind_cas(par, i, cap, err);
        if (r != i) vpar[i] = (uint16_t)r;
    }
    __syncthreads();
    // -- roots that own a pixel of the block border
    for (int j = t; j < PG::kEdge; j += T) {
        int row, col;
        border_pos<PG>(j, row, col);
        if ((sm.m[row][col >> 5] >> (col & 31)) & 1u) {
            const int i = piece_at<PG>(sm.S, sm.pb, sm.bb, row >> 1, col);
            const int r = proot1(vpar, i);
            atomicOr(&sm.border[r >> 5], 1u << (r & 31));
        }
    }
    __syncthreads();
    {
        // exclusive popcount prefix over the bitmap: kWPT words per thread,
        // then a scan over threads
        constexpr int kWPT = (kBorderWords + T - 1) / T;
        uint32_t c[kWPT], sum = 0;
#pragma unroll
        for (int q = 0; q < kWPT; ++q) {
            const int word = kWPT * t + q;
            c[q] = word < kBorderWords ? __popc(sm.border[word]) : 0u;
            sum += c[q];
        }
        uint32_t incl = sum;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t v = __shfl_up_sync(kFull, incl, d);
            if (lane >= d) incl += v;
        }
        if (lane == 31) sm.warp_tot[warp] = incl;
        __syncthreads();
        uint32_t base = 0;
        for (int q = 0; q < warp; ++q) base += sm.warp_tot[q];
        uint32_t run = base + incl - sum;
#pragma unroll
        for (int q = 0; q < kWPT; ++q) {
            const int word = kWPT * t + q;
            if (word < kBorderWords) sm.prefix[word] = run;
            run += c[q];
        }
        // at most kSlots border components exist; more marks only after an
        // iteration cap was hit, and the surplus slots are dropped
        if (t == T - 1) {
            sm.nslots = (int)(base + incl) < PG::kSlots ? (int)(base + incl) : PG::kSlots;
            if ((int)(base + incl) > PG::kSlots) sm.err |= kErrLocalCap;
        }
    }
    __syncthreads();
    // -- one global union-find entry per border component, keyed by its
    // minimum global raster position (ID conversion, Sec. 3.1.4)
    {
        const uint32_t sbase = b * (uint32_t)PG::kSlots;
        for (int word = t; word < kBorderWords; word += T) {
            uint32_t bits = sm.border[word];
            uint32_t slot = sm.prefix[word];
            for (; bits && slot < (uint32_t)PG::kSlots; bits &= bits - 1, ++slot) {
                const int at = word * 32 + lobit(bits);
                const int key = vpar[at] & 0x7FFF;
                const uint32_t g = job.key0 + (uint32_t)(y0 + (key >> PG::kBWLog2)) * (uint32_t)Wd +
                                   (uint32_t)(x0 + (key & (PG::kBW - 1)));
                s.P[sbase + slot] = pack_slot(g, sbase + slot);
                // from here on the root's entry is its slot (kBorderRoot | slot)
                vpar[at] = (uint16_t)(kBorderRoot | slot);
            }
        }
    }
    __syncthreads();
    // -- border record (slot of every border pixel), per-piece values, masks
    uint16_t *const Eb = s.edges + (size_t)b * PG::kEdge;
    for (int j = t; j < PG::kEdge; j += T) {
        int row, col;
        border_pos<PG>(j, row, col);
        uint16_t v = kBg;
        if ((sm.m[row][col >> 5] >> (col & 31)) & 1u)
            v = border_slot(pvalue(vpar, piece_at<PG>(sm.S, sm.pb, sm.bb, row >> 1, col)));
        Eb[j] = v;
    }
    uint16_t *const vout = s.values + (size_t)b * PG::kMaxPieces;
    for (int i = t; i < n; i += T) vout[i] = pvalue(vpar, i);
    {
        uint4 *mo = reinterpret_cast<uint4 *>(s.masks + (size_t)b * PG::kBH * W);
        const uint4 *mi = reinterpret_cast<const uint4 *>(&sm.m[0][0]);
        for (int q = t; q < PG::kBH * W / 4; q += T) mo[q] = mi[q];
    }
    if (err) atomicOr(&sm.err, err);
    __syncthreads();
    if (t == 0) {
        s.nslots[b] = sm.nslots;
        report(sm.err);
    }
}

template <class PG>
__global__ void __launch_bounds__(PG::kThreads, 5) k_piece_local(JobTable jt, PScratch s, int cap) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    PLocalSmem<PG> &sm = *reinterpret_cast<PLocalSmem<PG> *>(smem_raw);
    for (unsigned iter = 0; claim_item(jt, 0, iter, sm.item); ++iter) {
        const Job &job = sm.item.job;
        process_plocal<PG>(job, sm.item.lb, sm.item.gb, s, sm, cap);
        __syncthreads();
    }
    // when this grid was chained behind the previous labelling's write-out,
    // it ends only after that kernel (no-op otherwise): whatever runs after
    // this grid also runs after it
    grid_dependency_wait();
    // the merge may be launched now (it waits for this grid's completion)
    grid_launch_dependents();
}

// ---------------------------------------------------------------------------
// Step 3 (Sec. 3.3) on the piece layout.
template <class PG>
struct PWriteSmem {
    uint32_t m[PG::kBH][PG::kWords];
    uint32_t S[PG::kBands][PG::kWords];
    uint16_t pb[PG::kBands][PG::kWords];
    uint16_t bandcnt[PG::kBands];
    uint16_t bb[PG::kBands + 1];
    int slot_label[PG::kSlots];
    int lab[PG::kLabWindow];  // labels of the pieces of the current window of bands
    ItemSlot item;
};

// The labels of step 3 from the piece index tables of the block (row masks
// m, starts S, word prefixes pb, band prefix bb) with the buffers slot_label
// [kSlots] and lab [kLabWindow]; every thread of the CTA takes part.
template <class PG>
__device__ __forceinline__ void pwrite_labels(const Job &job, unsigned lb, unsigned gb, const PScratch &s,
                                              uint32_t (*m)[PG::kWords], const uint32_t (*S)[PG::kWords],
                                              uint16_t (*pb)[PG::kWords], const uint16_t *bb, int *slot_label,
                                              int *lab, int cap, uint32_t bound) {
    constexpr int W = PG::kWords;
    constexpr int T = PG::kThreads;
    constexpr int kChunks = PG::kBW / 4;  // 4-column chunks per row
    const unsigned b = gb;
    const int bx = (int)(lb % (unsigned)job.nbx), by = (int)(lb / (unsigned)job.nbx);
    const int H = job.H, Wd = job.W;
    int32_t *const labels = job.labels;
    const bool vec_out = (job.flags & kJobVecOut) != 0;
    const uint32_t key0 = job.key0;
    const int x0 = bx * PG::kBW, y0 = by * PG::kBH;
    const int t = threadIdx.x;
    // pb[k][w] becomes the index of the first piece of band k starting in word w or later
#pragma unroll
    for (int j = 0; j < PG::kBands * W / T; ++j) {
        const int item = t + j * T;
        const int k = item >> PG::kWordsLog2, w = item & (W - 1);
        pb[k][w] = (uint16_t)(pb[k][w] + bb[k]);
    }
    // a window of whole bands from band k0 whose piece labels fit in shared
    // memory: bands k0 .. k1 - 1
    const auto window_end = [&](int k0) {
        int k1 = k0 + 1;
        while (k1 < PG::kBands && (int)bb[k1 + 1] - (int)bb[k0] <= PG::kLabWindow) ++k1;
        return k1;
    };
    const uint16_t *const vin = s.values + (size_t)b * PG::kMaxPieces;
    // the values of the first window come from step 1 alone: they are read
    // before the wait below
    const int np_first = (int)bb[window_end(0)];
    for (int i = t; i < np_first; i += T) lab[i] = vin[i];
    // the merge (step 2) may still be running when this kernel starts
    // (programmatic dependent launch): wait for it before the first read of
    // the merged union-find
    grid_dependency_wait();
    // final label of each border slot: root-find in the merged union-find
    // (read-only; every union is complete after the wait)
    const int ns = s.nslots[b];
    int err = 0;
    for (int k = t; k < ns; k += T) {
        uint32_t key;
        find_global_ro(s.P, b * (uint32_t)PG::kSlots + (uint32_t)k, key, cap, err, bound);
        slot_label[k] = (int)key + 1;
    }
    report(err);
    __syncthreads();

    for (int k0 = 0; k0 < PG::kBands;) {
        const int k1 = window_end(k0);
        const int p0 = bb[k0], np = (int)bb[k1] - p0;
        for (int i = t; i < np; i += T) {
            // (the first window's values were loaded into lab by this thread)
            const uint32_t v = k0 == 0 ? (uint32_t)lab[i] : (uint32_t)vin[p0 + i];
            const uint32_t slot = v & 0x7FFFu;
            lab[i] = (v & kBorderFlag) ? ((int)slot < ns ? slot_label[slot] : 0)
                                          : (int)(key0 + (uint32_t)(y0 + (int)(v >> PG::kBWLog2)) * (uint32_t)Wd +
                                                  (uint32_t)(x0 + (int)(v & (PG::kBW - 1)))) + 1;
        }
        __syncthreads();
        // every pixel takes the label of its piece: a thread keeps one
        // 4-column chunk and walks down the bands of the window (a warp
        // writes 128 consecutive columns of two rows per step)
        {
            constexpr int kStep = T / kChunks;  // bands per step
            const int q = t & (kChunks - 1);
            const int w = q >> 3, c0 = (q & 7) * 4;
            const int x = x0 + 4 * q;
            const bool vec = vec_out && x + 4 <= Wd;
            const uint32_t below = (1u << c0) - 1u;
            if (x < Wd) {
                for (int k = k0 + t / kChunks; k < k1; k += kStep) {
                    const int y = y0 + 2 * k;
                    if (y >= H) break;
                    const uint32_t A4 = (m[2 * k][w] >> c0) & 15u, B4 = (m[2 * k + 1][w] >> c0) & 15u;
                    const uint32_t O4 = A4 | B4;
                    int l0 = 0, l1 = 0, l2 = 0, l3 = 0;
                    if (O4) {
                        const uint32_t Sw = S[k][w] >> c0;
                        const int idx = (int)pb[k][w] - p0 - 1 + __popc(S[k][w] & below);
                        const int i0 = idx + (int)(Sw & 1u), i1 = i0 + (int)((Sw >> 1) & 1u);
                        const int i2 = i1 + (int)((Sw >> 2) & 1u), i3 = i2 + (int)((Sw >> 3) & 1u);
                        if (O4 & 1u) l0 = lab[i0];
                        if (O4 & 2u) l1 = lab[i1];
                        if (O4 & 4u) l2 = lab[i2];
                        if (O4 & 8u) l3 = lab[i3];
                    }
                    int32_t *dst = labels + (size_t)y * Wd + x;
                    const int4 va = make_int4((A4 & 1u) ? l0 : 0, (A4 & 2u) ? l1 : 0, (A4 & 4u) ? l2 : 0,
                                              (A4 & 8u) ? l3 : 0);
                    const int4 vb = make_int4((B4 & 1u) ? l0 : 0, (B4 & 2u) ? l1 : 0, (B4 & 4u) ? l2 : 0,
                                              (B4 & 8u) ? l3 : 0);
                    const bool row2 = y + 1 < H;
                    if (vec) {
                        __stcs(reinterpret_cast<int4 *>(dst), va);
                        if (row2) __stcs(reinterpret_cast<int4 *>(dst + Wd), vb);
                    } else {
                        const int n = Wd - x < 4 ? Wd - x : 4;
                        const int a[4] = {va.x, va.y, va.z, va.w}, bq[4] = {vb.x, vb.y, vb.z, vb.w};
                        for (int e = 0; e < n; ++e) {
                            __stcs(dst + e, a[e]);
                            if (row2) __stcs(dst + Wd + e, bq[e]);
                        }
                    }
                }
            }
        }
        k0 = k1;
        __syncthreads();
    }
}


template <class PG>
__device__ __forceinline__ void process_pwrite(const Job &job, unsigned lb, unsigned gb, const PScratch &s,
                                               PWriteSmem<PG> &sm, int cap, uint32_t bound) {
    constexpr int W = PG::kWords;
    constexpr int T = PG::kThreads;
    const unsigned b = gb;
    const int t = threadIdx.x;
    {
        const uint4 *mi = reinterpret_cast<const uint4 *>(s.masks + (size_t)b * PG::kBH * W);
        uint4 *mo = reinterpret_cast<uint4 *>(&sm.m[0][0]);
        for (int q = t; q < PG::kBH * W / 4; q += T) mo[q] = mi[q];
    }
    // the piece index tables, from step 1's outputs only (step 1 finished
    // before the merge started)
    __syncthreads();
    band_tables<PG, false, false>(sm.m, sm.S, nullptr, nullptr, sm.pb, sm.bandcnt);
    __syncthreads();
    band_prefix<PG>(sm.bandcnt, sm.bb);
    __syncthreads();
    pwrite_labels<PG>(job, lb, gb, s, sm.m, sm.S, sm.pb, sm.bb, sm.slot_label, sm.lab, cap, bound);
}

template <class PG>
__global__ void __launch_bounds__(PG::kThreads, 7) k_piece_write(JobTable jt, PScratch s, int cap, uint32_t bound) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    PWriteSmem<PG> &sm = *reinterpret_cast<PWriteSmem<PG> *>(smem_raw);
    // a chained step 1 of the next labelling on the stream may start now: it
    // writes another scratch and finishes only after this grid
    grid_launch_dependents();
    for (unsigned iter = 0; claim_item(jt, 2, iter, sm.item); ++iter) {
        const Job &job = sm.item.job;
        process_pwrite<PG>(job, sm.item.lb, sm.item.gb, s, sm, cap, bound);
        __syncthreads();
    }
}

// The three steps in one cooperative grid, for images whose blocks can all be
// resident at once (one block per CTA): step 1, a grid-wide barrier, the
// block's merge, a barrier, then the write-out from the piece index tables
// step 1 left in shared memory (no reload of the masks, no second table
// build, no kernel boundaries).  The merge and the write-out buffers overlay
// step 1's candidate list and equivalence list, which are dead by then.
template <class PG>
__global__ void __launch_bounds__(PG::kThreads, 5) k_piece_coop(JobTable jt, PScratch s, int cap, Scratch ms,
                                                                int gcap, uint32_t bound) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    PLocalSmem<PG> &sm = *reinterpret_cast<PLocalSmem<PG> *>(smem_raw);
    constexpr size_t kOverlay = offsetof(PLocalSmem<PG>, border) - offsetof(PLocalSmem<PG>, cand);
    static_assert(sizeof(MergeSmem<PG>) <= kOverlay, "merge overlay");
    static_assert((PG::kSlots + PG::kLabWindow) * sizeof(int) <= kOverlay, "write-out overlay");
    cooperative_groups::grid_group grid = cooperative_groups::this_grid();
    claim_item(jt, 0, 0, sm.item);  // block blockIdx.x of the single image
    const Job &job = sm.item.job;
    const unsigned lb = sm.item.lb, gb = sm.item.gb;
    process_plocal<PG>(job, lb, gb, s, sm, cap);
    grid.sync();
    MergeSmem<PG> &msm = *reinterpret_cast<MergeSmem<PG> *>(sm.cand);
    process_merge<PG, PG::kConn8, true>(job, lb, gb, ms, msm, cap, gcap, bound);
    grid.sync();
    int *const slot_label = reinterpret_cast<int *>(sm.cand);
    pwrite_labels<PG>(job, lb, gb, s, sm.m, sm.S, sm.pb, sm.bb, slot_label, slot_label + PG::kSlots, cap, bound);
}

}  // namespace ccl
