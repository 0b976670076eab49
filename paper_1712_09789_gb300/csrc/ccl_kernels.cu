// ccl_kernels.cu -- the three steps of the block-based labeller as sm_103a
// kernels, and the launchers that enqueue them on a stream.
//
//   k_block_local   step 1, Kernel 1 (Sec. 3.1) on blocks of 32*BLX x 8*BLY
//                   pixels: every thread labels its 32 x 8 lane tile by coarse
//                   labelling (row connection by bit operations; column
//                   connection to the first run above) and refinement (merging
//                   the further runs above); the lane tiles of the block are
//                   then merged along their seams.  Writes the block's row
//                   masks, one value per run (block key of its root, or its
//                   border slot), the border record of the block and one
//                   global union-find entry per border component.
//   k_block_merge   step 2, Kernel 2 (Sec. 3.2, Eq. 1-2): only the pixel
//                   pairs that straddle a block edge are examined.
//   k_block_write   step 3 (Sec. 3.3): root-find for the block's border slots
//                   in the merged union-find, then expands the per-run values
//                   over the row masks and writes every label once.
//
// Work items are blocks.  A single image launches one CTA per block; a batch
// of images launches persistent CTAs that take blocks from a device counter
// and find each block's image in a job table (blocks of an image are
// consecutive items, in raster order).
//
// HBM traffic per pixel: 1 B image read, 4 B label write, plus the row masks
// (1/8 B written, 1/8 B read) and the per-run values (1 B label and 2 B value
// per run, written and read once), most of which stay in L2.
#include <algorithm>
#include <cstdint>
#include <deque>
#include <mutex>
#include <vector>

#include <cuda_runtime.h>

#include "ccl_block.cuh"
#include "ccl_internal.h"

namespace ccl {

__device__ int g_device_error = 0;

// Per-block scratch regions, indexed by the global block (item) index; sized
// for capacity, only the used parts are touched.
struct Scratch {
    uint32_t *masks;   // [blocks][threads][8 rows]
    uint32_t *lstream; // [blocks][kLWords][threads]: run labels, 4 per word
    uint4 *vstream;    // [blocks][kVChunks][threads]: run values, 8 per chunk
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
template <class G>
struct LocalSmem {
    uint16_t par[kLabCap * G::kThreads];           // list entries, see ccl_block.cuh
    uint8_t lab[3][kLW][G::kLabPitch];             // run-start labels: row 0, then two alternating rows
    uint8_t lcol[kLH][G::kLabPitch];               // label of the run holding column 0, per row
    uint8_t rcol[kLH][G::kLabPitch];               // label of the run holding column 31, per row
    uint32_t mask[kLH][G::kThreads];               // row masks
    union {
        uint16_t qpair[16][G::kThreads];           // further contacts of the current row (scan)
        struct {
            uint32_t border[kLabCap * G::kThreads / 32];  // bit per id: root touching the block border
            uint32_t prefix[kLabCap * G::kThreads / 32];
        };
    };
    uint32_t warp_tot[G::kThreads / 32];
    int nslots;
    int err;
    ItemSlot item;
};

__device__ __forceinline__ int lab_buf(int r) { return r == 0 ? 0 : 1 + ((r - 1) & 1); }

// Border record entry of a run value: its slot, or background when the value
// is not a border slot (only possible after an iteration cap was hit).
__device__ __forceinline__ uint16_t border_slot(uint16_t v) {
    return (v & kBorderFlag) ? (uint16_t)(v & 0x3FFF) : kBg;
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

template <class G, bool kConn8>
__device__ __forceinline__ void process_local(const Job &job, unsigned lb, unsigned gb, const Scratch &s,
                                              LocalSmem<G> &sm, int cap) {

    const unsigned b = gb;
    const int bx = (int)(lb % (unsigned)job.nbx), by = (int)(lb / (unsigned)job.nbx);
    const int H = job.H, W = job.W;
    const uint8_t *const img = job.img;
    const size_t pitch = (size_t)job.pitch;
    const bool vec_in = (job.flags & kJobVecIn) != 0;
    const int x0 = bx * G::kBW, y0 = by * G::kBH;
    const int t = threadIdx.x;
    const int tx = t & (G::BLX - 1), ty = t >> G::kBLXLog2;
    const int xl = x0 + kLW * tx, yl = y0 + kLH * ty;
    int err = 0;

    if (t == 0) sm.err = 0;
    __syncthreads();

    // -- initialization: the lane tile's 8 rows as masks (all loads in flight
    // at once; pixels outside the image are background)
    uint32_t mrow[kLH];
    if (vec_in && xl + kLW <= W && yl + kLH <= H) {
        uint4 raw[2 * kLH];
        const uint8_t *p = img + (size_t)yl * pitch + xl;
#pragma unroll
        for (int r = 0; r < kLH; ++r) {
            raw[2 * r] = ldg_nc16(p + (size_t)r * pitch);
            raw[2 * r + 1] = ldg_nc16(p + (size_t)r * pitch + 16);
        }
#pragma unroll
        for (int r = 0; r < kLH; ++r) mrow[r] = nz16(raw[2 * r]) | (nz16(raw[2 * r + 1]) << 16);
    } else {
#pragma unroll
        for (int r = 0; r < kLH; ++r) {
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
    for (int r = 0; r < kLH; ++r) sm.mask[r][t] = mrow[r];

    // -- coarse labelling and refinement, row by row.  Every loop below runs
    // the same number of rounds on all 32 lanes of a warp (the maximum any
    // lane needs), so the 32 lane tiles advance in lockstep.
    //
    // Coarse labelling: a run with foreground above takes the label value of
    // the first run above it (row connection by bit operations, column
    // connection to that run); labels therefore travel down unchanged and
    // no list is walked here.  A run without foreground above opens a new
    // list.  Refinement: every further run above that a run touches is
    // queued and the queued pairs of the row are merged after the row, the
    // larger root hung under the smaller.
    volatile uint16_t *vpar = sm.par;
    uint32_t prevM = 0, prevS = 0;
    int nlab = 0, nrun = 0;
    uint32_t lacc = 0;                              // 4 run labels, first in the low byte
    uint32_t *lout = s.lstream + (size_t)b * kLWords * G::kThreads + t;
#pragma unroll 1
    for (int r = 0; r < kLH; ++r) {
        const uint32_t m = sm.mask[r][t];
        uint32_t S = m & ~(m << 1);                 // run starts
        uint32_t E = m & ~(m >> 1);                 // run ends
        uint8_t *cur = &sm.lab[lab_buf(r)][0][t];
        const uint8_t *prev = &sm.lab[lab_buf(r > 0 ? r - 1 : 0)][0][t];
        int nq = 0;
        const int nmax = __reduce_max_sync(kFull, __popc(S));
        for (int k = 0; k < nmax; ++k) {
            const bool act = S != 0u;
            // an exhausted lane sees a dummy run at bit 31 and stores nothing
            const int a0 = lobit(S | 0x80000000u);
            const int a1 = lobit(E | 0x80000000u);
            S &= S - 1u;
            E &= E - 1u;
            const uint32_t P = prevM & touch_range<kConn8>(run_bits(a0, a1)) & (0u - (uint32_t)act);
            const int u0 = P ? lobit(P) : 0;
            int L = nlab;
            if (P) L = prev[hibit(prevS & upto(u0)) * G::kLabPitch];
            else if (act) {
                vpar[nlab * G::kThreads + t] = (uint16_t)(kRoot | (r * kLW + a0));
                ++nlab;
            }
            uint32_t Q = P ? (prevS & P & ~upto(u0)) : 0u;
            while (__any_sync(kFull, Q != 0u)) {
                if (Q) {
                    sm.qpair[nq][t] = (uint16_t)(L | (prev[lobit(Q) * G::kLabPitch] << 8));
                    ++nq;
                    Q &= Q - 1u;
                }
            }
            if (act) {
                cur[a0 * G::kLabPitch] = (uint8_t)L;
                lacc = (lacc >> 8) | ((uint32_t)L << 24);
                ++nrun;
                if ((nrun & 3) == 0) lout[(size_t)((nrun >> 2) - 1) * G::kThreads] = lacc;
            }
        }
        sm.lcol[r][t] = (m & 1u) ? cur[0] : (uint8_t)0xFF;
        sm.rcol[r][t] = (m >> 31) ? cur[hibit(m & ~(m << 1)) * G::kLabPitch] : (uint8_t)0xFF;
        prevM = m;
        prevS = m & ~(m << 1);
        // refinement of the row: merge the queued pairs (own lists only)
        const int nqmax = __reduce_max_sync(kFull, nq);
        for (int j = 0; j < nqmax; ++j) {
            const bool hq = j < nq;
            const uint16_t pr = hq ? sm.qpair[j][t] : (uint16_t)0;
            int A = pr & 0xFF, B = pr >> 8;
            bool pa = hq, pb = hq;
            for (int i = 0; __any_sync(kFull, pa || pb); ++i) {
                // root-finds with path halving (own lists, no other writer)
                if (pa) {
                    const uint16_t e = vpar[A * G::kThreads + t];
                    if (e & kRoot) {
                        pa = false;
                    } else {
                        const int p = e & (kLabCap - 1);
                        const uint16_t g = vpar[p * G::kThreads + t];
                        if (g & kRoot) { A = p; pa = false; }
                        else { vpar[A * G::kThreads + t] = g; A = g & (kLabCap - 1); }
                    }
                }
                if (pb) {
                    const uint16_t e = vpar[B * G::kThreads + t];
                    if (e & kRoot) {
                        pb = false;
                    } else {
                        const int p = e & (kLabCap - 1);
                        const uint16_t g = vpar[p * G::kThreads + t];
                        if (g & kRoot) { B = p; pb = false; }
                        else { vpar[B * G::kThreads + t] = g; B = g & (kLabCap - 1); }
                    }
                }
                if (i >= cap) {
                    if (pa || pb) err |= kErrLocalCap;
                    break;
                }
            }
            if (hq && A != B) {
                const int lo = A < B ? A : B, hi = A < B ? B : A;
                vpar[hi * G::kThreads + t] = (uint16_t)lo;
            }
        }
        __syncwarp();
    }
    if (nrun & 3) lout[(size_t)(nrun >> 2) * G::kThreads] = lacc >> (8 * (4 - (nrun & 3)));
    // compress the own lists (labels are still lane-local here, so no other
    // lane reads them) and turn parent links into block-wide ids: the thread
    // index joins the label
    const int nlab_max = __reduce_max_sync(kFull, nlab);
    for (int L = 0; L < nlab_max; ++L) {
        if (L < nlab) {
            // entries already converted by earlier rounds carry this thread's
            // index in their high bits; the low bits are the lane-local label
            int x = L;
            uint16_t e = vpar[x * G::kThreads + t];
            for (int i = 0; !(e & kRoot) && i < cap; ++i) {
                x = e & (kLabCap - 1);
                e = vpar[x * G::kThreads + t];
            }
            if (x != L) vpar[L * G::kThreads + t] = (uint16_t)((t << 7) | x);
        }
    }
    __syncthreads();

    // the refinement queue is dead now; its space holds the border bitmap
    for (int i = t; i < kLabCap * G::kThreads / 32; i += G::kThreads) sm.border[i] = 0u;

    // -- block merge of the lane tiles along their seams (Kernel 2's boundary
    // analysis applied inside the block, on the shared lists)
    const uint32_t m0 = mrow[0];
    {
        const bool hasl = tx > 0;
        const int tl = hasl ? t - 1 : t;
#pragma unroll
        for (int r = 0; r < kLH; ++r) {
            const bool me_fg = hasl && (mrow[r] & 1u);
            const int me = (t << 7) | sm.lcol[r][t];
            // a pair repeating the row above's pair (both columns continue
            // vertically) adds nothing
            const bool up_me = r > 0 && (mrow[r > 0 ? r - 1 : 0] & 1u);
            const bool dn_me = r + 1 < kLH && (mrow[r + 1 < kLH ? r + 1 : r] & 1u);
            const bool up_l = r > 0 && (sm.mask[r > 0 ? r - 1 : 0][tl] >> 31);
            const bool dn_l = r + 1 < kLH && (sm.mask[r + 1 < kLH ? r + 1 : r][tl] >> 31);
            const bool at_l = sm.mask[r][tl] >> 31;
            union_block_sync<G>(sm.par, me_fg && at_l && !(up_me && up_l), me, (tl << 7) | sm.rcol[r][tl], cap, err);
            if (kConn8) {
                union_block_sync<G>(sm.par, me_fg && up_l && !up_me, me,
                                 (tl << 7) | sm.rcol[r > 0 ? r - 1 : 0][tl], cap, err);
                union_block_sync<G>(sm.par, me_fg && dn_l && !dn_me, me,
                                 (tl << 7) | sm.rcol[r + 1 < kLH ? r + 1 : r][tl], cap, err);
            }
        }
    }
    {
        const bool hasu = ty > 0;
        const int tu = hasu ? t - G::BLX : t;
        const uint32_t mU = hasu ? sm.mask[kLH - 1][tu] : 0u;
        const uint32_t SU = mU & ~(mU << 1);
        const uint8_t *top = &sm.lab[0][0][t];
        const uint8_t *bot = &sm.lab[lab_buf(kLH - 1)][0][tu];
        uint32_t S = hasu ? (m0 & ~(m0 << 1)) : 0u;
        uint32_t E = m0 & ~(m0 >> 1);
        const int nmax = __reduce_max_sync(kFull, __popc(S));
        for (int k = 0; k < nmax; ++k) {
            const bool act = S != 0u;
            const int a0 = act ? lobit(S) : 0;
            const int a1 = act ? lobit(E) : 0;
            S &= S - 1u;
            E &= E - 1u;
            const uint32_t P = act ? (mU & touch_range<kConn8>(run_bits(a0, a1))) : 0u;
            const int me = (t << 7) | top[a0 * G::kLabPitch];
            const int u0 = P ? lobit(P) : 0;
            union_block_sync<G>(sm.par, P != 0u, me, (tu << 7) | bot[hibit((SU & upto(u0)) | 1u) * G::kLabPitch], cap,
                             err);
            uint32_t Q = P ? (SU & P & ~upto(u0)) : 0u;
            while (__any_sync(kFull, Q != 0u)) {
                const bool hq = Q != 0u;
                const int q = hq ? lobit(Q) : 0;
                Q &= Q - 1u;
                union_block_sync<G>(sm.par, hq, me, (tu << 7) | bot[q * G::kLabPitch], cap, err);
            }
        }
        if (kConn8) {
            // corners: the lane tiles up-left and up-right
            const bool ul = hasu && tx > 0 && (m0 & 1u);
            const int tul = ul ? tu - 1 : t;
            const uint32_t mUL = ul ? sm.mask[kLH - 1][tul] : 0u;
            const uint32_t SUL = mUL & ~(mUL << 1);
            union_block_sync<G>(sm.par, ul && (mUL >> 31), (t << 7) | top[0],
                             (tul << 7) | sm.lab[lab_buf(kLH - 1)][hibit(SUL | 1u)][tul], cap, err);
            const bool ur = hasu && tx + 1 < G::BLX && (m0 >> 31);
            const int tur = ur ? tu + 1 : t;
            const uint32_t S0 = m0 & ~(m0 << 1);
            union_block_sync<G>(sm.par, ur && (sm.mask[kLH - 1][tur] & 1u), (t << 7) | top[hibit(S0 | 1u) * G::kLabPitch],
                             (tur << 7) | sm.lab[lab_buf(kLH - 1)][0][tur], cap, err);
        }
    }
    __syncthreads();

    // -- compress: every own list entry points straight at its root (the
    // finds only read, so every store here is a final root)
    for (int L = 0; L < nlab_max; ++L) {
        if (L < nlab) {
            const int id = (t << 7) | L;
            const int root = find_root_ro<G>(vpar, id, cap, err);
            if (root != id) vpar[L * G::kThreads + t] = (uint16_t)root;
        }
    }
    __syncthreads();

    // -- roots that own a pixel of the block border
    auto root_of = [&](int id) -> int {
        const uint16_t e = vpar[par_index<G>(id)];
        return (e & kRoot) ? id : (int)e;
    };
    auto mark = [&](int id) {
        const int root = root_of(id);
        atomicOr(&sm.border[root >> 5], 1u << (root & 31));
    };
    if (ty == 0)
        for (uint32_t S = m0 & ~(m0 << 1); S; S &= S - 1) mark((t << 7) | sm.lab[0][lobit(S)][t]);
    if (ty == G::BLY - 1) {
        const uint32_t m7 = mrow[kLH - 1];
        for (uint32_t S = m7 & ~(m7 << 1); S; S &= S - 1)
            mark((t << 7) | sm.lab[lab_buf(kLH - 1)][lobit(S)][t]);
    }
    if (tx == 0) {
#pragma unroll
        for (int r = 0; r < kLH; ++r)
            if (mrow[r] & 1u) mark((t << 7) | sm.lcol[r][t]);
    }
    if (tx == G::BLX - 1) {
#pragma unroll
        for (int r = 0; r < kLH; ++r)
            if (mrow[r] >> 31) mark((t << 7) | sm.rcol[r][t]);
    }
    __syncthreads();
    {
        // exclusive popcount prefix over 512 words: 4 per thread, then a scan
        uint32_t c[4], sum = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) { c[k] = __popc(sm.border[4 * t + k]); sum += c[k]; }
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
        for (int k = 0; k < 4; ++k) { sm.prefix[4 * t + k] = run; run += c[k]; }
        // at most G::kSlots border components exist; more marks only after an
        // iteration cap was hit, and the surplus slots are dropped
        if (t == G::kThreads - 1) {
            sm.nslots = (int)(base + incl) < G::kSlots ? (int)(base + incl) : G::kSlots;
            if ((int)(base + incl) > G::kSlots) sm.err |= kErrLocalCap;
        }
    }
    __syncthreads();
    auto slot_of = [&](int root) -> int {
        return (int)(sm.prefix[root >> 5] + __popc(sm.border[root >> 5] & ((1u << (root & 31)) - 1u)));
    };

    // -- one global union-find entry per border component, keyed by its
    // minimum global raster position (ID conversion, Sec. 3.1.4)
    {
        const uint32_t sbase = (uint32_t)b * G::kSlots;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int word = 4 * t + k;
            uint32_t bits = sm.border[word];
            uint32_t slot = sm.prefix[word];
            for (; bits && slot < (uint32_t)G::kSlots; bits &= bits - 1, ++slot) {
                const int root = word * 32 + lobit(bits);
                const int key = root_key<G>(root, vpar[par_index<G>(root)]);
                const uint32_t g = (uint32_t)(y0 + (key >> G::kBWLog2)) * (uint32_t)W +
                                   (uint32_t)(x0 + (key & (G::kBW - 1)));
                s.P[sbase + slot] = pack_slot(g, sbase + slot);
            }
        }
    }
    __syncthreads();
    // -- each own root entry becomes the value its runs carry from now on
    for (int L = 0; L < nlab_max; ++L) {
        if (L < nlab) {
            const int id = (t << 7) | L;
            const uint16_t e = vpar[L * G::kThreads + t];
            if (e & kRoot) {
                const bool border = (sm.border[id >> 5] >> (id & 31)) & 1u;
                vpar[L * G::kThreads + t] = border ? (uint16_t)(kRootBorder | slot_of(id))
                                                : (uint16_t)(kRoot | root_key<G>(id, e));
            }
        }
    }
    __syncthreads();
    // ... and so does every own non-root entry (it points straight at a root,
    // whose value is final), making a run's value a single lookup
    for (int L = 0; L < nlab_max; ++L) {
        if (L < nlab) {
            const uint16_t e = vpar[L * G::kThreads + t];
            if (e < kRootBorder) vpar[L * G::kThreads + t] = vpar[par_index<G>(e)];
        }
    }

    // -- border record of the block: the slot of every border pixel
    uint16_t *Eb = s.edges + (size_t)b * G::kEdge;
    if (ty == 0 || ty == G::BLY - 1) {
        const int rr = ty == 0 ? 0 : kLH - 1;
        const uint32_t m = mrow[rr];
        const uint32_t S = m & ~(m << 1);
        const uint8_t *lb = &sm.lab[lab_buf(rr)][0][t];
        uint16_t *dst = Eb + (ty == 0 ? G::kEdgeTop : G::kEdgeBottom) + kLW * tx;
#pragma unroll 4
        for (int c = 0; c < kLW; ++c) {
            uint16_t v = kBg;
            if ((m >> c) & 1u) v = border_slot(run_value<G>(vpar, (t << 7) | lb[hibit(S & upto(c)) * G::kLabPitch]));
            dst[c] = v;
        }
    }
    if (tx == 0 || tx == G::BLX - 1) {
        uint16_t *dst = Eb + (tx == 0 ? G::kEdgeLeft : G::kEdgeRight) + kLH * ty;
#pragma unroll
        for (int r = 0; r < kLH; ++r) {
            const bool fg = tx == 0 ? (mrow[r] & 1u) : (mrow[r] >> 31);
            const int L = tx == 0 ? sm.lcol[r][t] : sm.rcol[r][t];
            dst[r] = fg ? border_slot(run_value<G>(vpar, (t << 7) | L)) : kBg;
        }
    }
    // -- per-run values: block key of the root, or kBorderFlag | slot
    {
        const uint32_t *lin = s.lstream + (size_t)b * kLWords * G::kThreads + t;
        uint4 *vout = s.vstream + (size_t)b * kVChunks * G::kThreads + t;
        HalfQueue vq;
        const int nrun_max = __reduce_max_sync(kFull, nrun);
        for (int k = 0; k < nrun_max; k += 4) {
            const uint32_t w = k < nrun ? lin[(size_t)(k >> 2) * G::kThreads] : 0u;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (k + j < nrun) {
                    vq.push(run_value<G>(vpar, (t << 7) | ((w >> (8 * j)) & 0xFF)));
                    if (((k + j + 1) & 7) == 0) vout[(size_t)((k + j) >> 3) * G::kThreads] = vq.bits();
                }
            }
        }
        if (nrun & 7) {
            for (int k = nrun & 7; k < 8; ++k) vq.push(0);
            vout[(size_t)(nrun >> 3) * G::kThreads] = vq.bits();
        }
    }
    // -- row masks for the write-out pass
    {
        uint4 *mo = reinterpret_cast<uint4 *>(s.masks + ((size_t)b * G::kThreads + t) * kLH);
        mo[0] = make_uint4(mrow[0], mrow[1], mrow[2], mrow[3]);
        mo[1] = make_uint4(mrow[4], mrow[5], mrow[6], mrow[7]);
    }
    if (err) atomicOr(&sm.err, err);
    __syncthreads();
    if (t == 0) {
        s.nslots[b] = sm.nslots;
        report(sm.err);
    }
}

template <class G, bool kConn8>
__global__ void __launch_bounds__(G::kThreads, 4) k_block_local(JobTable jt, Scratch s, int cap) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    LocalSmem<G> &sm = *reinterpret_cast<LocalSmem<G> *>(smem_raw);
    for (unsigned iter = 0; claim_item(jt, 0, iter, sm.item); ++iter) {
        const Job &job = sm.item.job;
        const unsigned lb = sm.item.lb, gb = sm.item.gb;
        process_local<G, kConn8>(job, lb, gb, s, sm, cap);
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Each block examines the pixel pairs across its top edge, its left edge and
// (8-connectivity) its two upper corners; the right, bottom and lower corners
// belong to the neighbouring blocks.  A pair that repeats the pair of the
// neighbouring pixel is skipped.  One thread per top-edge column.
template <class G, bool kConn8>
__device__ __forceinline__ void process_merge(const Job &job, unsigned lb, unsigned gb, const Scratch &s, int cap,
                                              uint32_t bound) {

    const unsigned b = gb;
    const int nbx = job.nbx;
    const int bx = (int)(lb % (unsigned)nbx), by = (int)(lb / (unsigned)nbx);
    const uint16_t *E = s.edges + (size_t)b * G::kEdge;
    const uint32_t base = (uint32_t)b * G::kSlots;
    int err = 0;
    // every slot named by a border record is below its block's slot count;
    // checking it keeps the finds inside initialised entries whatever happened
    const auto valid = [&](unsigned blk, uint16_t v) { return v != kBg && (int)v < s.nslots[blk]; };

    if (by > 0) {
        const unsigned bu = b - (unsigned)nbx;
        const uint16_t *Eu = s.edges + (size_t)bu * G::kEdge;
        const uint32_t ubase = (uint32_t)bu * G::kSlots;
        for (int j = threadIdx.x; j < G::kBW; j += G::kBW) {
            const uint16_t a = E[G::kEdgeTop + j];
            if (!valid(b, a)) continue;
            const uint16_t aL = j > 0 ? E[G::kEdgeTop + j - 1] : kBg;
            const uint16_t aR = j + 1 < G::kBW ? E[G::kEdgeTop + j + 1] : kBg;
            const uint16_t c = Eu[G::kEdgeBottom + j];
            const uint16_t cL = j > 0 ? Eu[G::kEdgeBottom + j - 1] : kBg;
            if (valid(bu, c) && !(aL == a && cL == c)) union_global(s.P, base + a, ubase + c, cap, err, bound);
            if (kConn8) {
                if (j > 0) {
                    if (valid(bu, cL) && aL != a) union_global(s.P, base + a, ubase + cL, cap, err, bound);
                } else if (bx > 0) {
                    const uint16_t d = s.edges[(size_t)(bu - 1) * G::kEdge + G::kEdgeBottom + G::kBW - 1];
                    if (valid(bu - 1, d)) union_global(s.P, base + a, (uint32_t)(bu - 1) * G::kSlots + d, cap, err, bound);
                }
                if (j + 1 < G::kBW) {
                    const uint16_t cR = Eu[G::kEdgeBottom + j + 1];
                    if (valid(bu, cR) && aR != a) union_global(s.P, base + a, ubase + cR, cap, err, bound);
                } else if (bx + 1 < nbx) {
                    const uint16_t d = s.edges[(size_t)(bu + 1) * G::kEdge + G::kEdgeBottom + 0];
                    if (valid(bu + 1, d)) union_global(s.P, base + a, (uint32_t)(bu + 1) * G::kSlots + d, cap, err, bound);
                }
            }
        }
    }
    if (bx > 0) {
        const unsigned bl = b - 1;
        const uint16_t *El = s.edges + (size_t)bl * G::kEdge;
        const uint32_t lbase = (uint32_t)bl * G::kSlots;
        for (int j = threadIdx.x; j < G::kBH; j += G::kBW) {
            const uint16_t a = E[G::kEdgeLeft + j];
            if (!valid(b, a)) continue;
            const uint16_t aU = j > 0 ? E[G::kEdgeLeft + j - 1] : kBg;
            const uint16_t aD = j + 1 < G::kBH ? E[G::kEdgeLeft + j + 1] : kBg;
            const uint16_t c = El[G::kEdgeRight + j];
            const uint16_t cU = j > 0 ? El[G::kEdgeRight + j - 1] : kBg;
            if (valid(bl, c) && !(aU == a && cU == c)) union_global(s.P, base + a, lbase + c, cap, err, bound);
            if (kConn8) {
                if (j > 0 && valid(bl, cU) && aU != a) union_global(s.P, base + a, lbase + cU, cap, err, bound);
                if (j + 1 < G::kBH) {
                    const uint16_t cD = El[G::kEdgeRight + j + 1];
                    if (valid(bl, cD) && aD != a) union_global(s.P, base + a, lbase + cD, cap, err, bound);
                }
            }
        }
    }
    report(err);
}

template <class G, bool kConn8>
__global__ void __launch_bounds__(G::kBW) k_block_merge(JobTable jt, Scratch s, int cap, uint32_t bound) {
    __shared__ ItemSlot item;
    for (unsigned iter = 0; claim_item(jt, 1, iter, item); ++iter) {
        const Job &job = item.job;
        const unsigned lb = item.lb, gb = item.gb;
        process_merge<G, kConn8>(job, lb, gb, s, cap, bound);
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
template <class G>
struct WriteSmem {
    int slot_label[G::kSlots];
    int runlab[G::BLY][G::kBW];          // label of every run at its start column, one row of all lane tiles
    uint32_t mask[kLH][G::kThreads];     // row masks of the block
    ItemSlot item;
};

// Position of (lane tile tx, column c) in a runlab row: the column is XORed
// with tx so that neighbouring lane tiles read by one warp of the copy-out
// spread over the banks.
template <class G>
__device__ __forceinline__ int runlab_index(int tx, int c) { return kLW * tx + (c ^ ((tx & 3) << 3)); }

template <class G>
__device__ __forceinline__ void process_write(const Job &job, unsigned lb, unsigned gb, const Scratch &s,
                                              WriteSmem<G> &sm, int cap, uint32_t bound) {

    const unsigned b = gb;
    const int bx = (int)(lb % (unsigned)job.nbx), by = (int)(lb / (unsigned)job.nbx);
    const int H = job.H, W = job.W;
    int32_t *const labels = job.labels;
    const bool vec_out = (job.flags & kJobVecOut) != 0;
    const int x0 = bx * G::kBW, y0 = by * G::kBH;
    const int t = threadIdx.x;
    const int tx = t & (G::BLX - 1), ty = t >> G::kBLXLog2;

    // final label of each border slot: root-find in the merged union-find
    // (read-only; every union is complete when this kernel starts)
    const int ns = s.nslots[b];
    int err = 0;
    for (int k = t; k < ns; k += G::kThreads) {
        uint32_t key;
        find_global_ro(s.P, (uint32_t)b * G::kSlots + (uint32_t)k, key, cap, err, bound);
        sm.slot_label[k] = (int)key + 1;
    }
    report(err);

    const uint4 *mi = reinterpret_cast<const uint4 *>(s.masks + ((size_t)b * G::kThreads + t) * kLH);
    const uint4 mA = mi[0], mB = mi[1];
    const uint32_t mrow[kLH] = {mA.x, mA.y, mA.z, mA.w, mB.x, mB.y, mB.z, mB.w};
#pragma unroll
    for (int r = 0; r < kLH; ++r) sm.mask[r][t] = mrow[r];
    // per-run values, 8 per chunk; the next chunk is always already in flight
    const uint4 *vin = s.vstream + (size_t)b * kVChunks * G::kThreads + t;
    int nrun = 0;
#pragma unroll
    for (int r = 0; r < kLH; ++r) nrun += __popc(mrow[r] & ~(mrow[r] << 1));
    const int nchunks = (nrun + 7) >> 3;
    uint4 vq = nchunks > 0 ? vin[0] : make_uint4(0, 0, 0, 0);
    uint4 vnext = nchunks > 1 ? vin[G::kThreads] : make_uint4(0, 0, 0, 0);
    int vi = 0, vc = 2;
    __syncthreads();

#pragma unroll
    for (int r = 0; r < kLH; ++r) {
        // each lane tile: one label per run of its row r, at the run start
        const uint32_t m = mrow[r];
        uint32_t S = m & ~(m << 1);
        const int nmax = __reduce_max_sync(kFull, __popc(S));
        for (int k = 0; k < nmax; ++k) {
            if (S) {
                const int a0 = lobit(S);
                S &= S - 1u;
                if (vi == 8) {
                    vq = vnext;
                    if (vc < nchunks) vnext = vin[(size_t)vc * G::kThreads];
                    ++vc;
                    vi = 0;
                }
                const uint32_t w = vi < 2 ? vq.x : vi < 4 ? vq.y : vi < 6 ? vq.z : vq.w;
                const uint32_t v = (w >> ((vi & 1) * 16)) & 0xFFFFu;
                ++vi;
                const uint32_t slot = v & 0x7FFFu;
                const int lab = (v & kBorderFlag) ? ((int)slot < ns ? sm.slot_label[slot] : 0)
                                                   : (int)((uint32_t)(y0 + (int)(v >> G::kBWLog2)) * (uint32_t)W +
                                                           (uint32_t)(x0 + (int)(v & (G::kBW - 1)))) + 1;
                sm.runlab[ty][runlab_index<G>(tx, a0)] = lab;
            }
        }
        __syncthreads();
        // coalesced write-out of image rows y0 + 8*ry + r: every pixel takes
        // the label stored at the start of its run; a thread covers 4 pixels
        // per step
        for (int i = t; i < G::BLY * (G::kBW / 4); i += G::kThreads) {
            const int ry = i / (G::kBW / 4);
            const int q = i % (G::kBW / 4);         // 4-pixel chunk of the row
            const int ctx = q >> 3;                 // its lane tile
            const int c0 = (q & 7) * 4;             // its first column in the lane tile
            const int x = x0 + 4 * q;
            const int y = y0 + kLH * ry + r;
            if (y < H && x < W) {
                const uint32_t mm = sm.mask[r][ry * G::BLX + ctx];
                const uint32_t SS = mm & ~(mm << 1);
                int v[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int c = c0 + j;
                    v[j] = ((mm >> c) & 1u) ? sm.runlab[ry][runlab_index<G>(ctx, hibit(SS & upto(c)))] : 0;
                }
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

template <class G>
__global__ void __launch_bounds__(G::kThreads, 4) k_block_write(JobTable jt, Scratch s, int cap, uint32_t bound) {
    __shared__ WriteSmem<G> sm;
    for (unsigned iter = 0; claim_item(jt, 2, iter, sm.item); ++iter) {
        const Job &job = sm.item.job;
        const unsigned lb = sm.item.lb, gb = sm.item.gb;
        process_write<G>(job, lb, gb, s, sm, cap, bound);
        __syncthreads();
    }
}

}  // namespace ccl

// ---------------------------------------------------------------------------
// Host side of this translation unit.

namespace ccl {

namespace {

size_t up256(size_t v) { return (v + 255) & ~(size_t)255; }

struct Layout {
    size_t masks, lstream, vstream, edges, P, nslots, total;
};

template <class G>
Layout layout_for(size_t nb) {
    Layout l;
    size_t off = 0;
    l.masks = off;   off += up256(nb * G::kThreads * kLH * sizeof(uint32_t));
    l.lstream = off; off += up256(nb * kLWords * G::kThreads * sizeof(uint32_t));
    l.vstream = off; off += up256(nb * kVChunks * G::kThreads * sizeof(uint4));
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
    s.lstream = reinterpret_cast<uint32_t *>(p + l.lstream);
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

using G0 = Geo<16, 8>;
using G1 = Geo<8, 8>;
using G2 = Geo<32, 4>;

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
        if (r.kind == kKernelKinds - 1) g_timing.pool.push_back(r.b);
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
    static const char *names[kKernelKinds] = {"k_block_local", "k_block_merge", "k_block_write"};
    return (k >= 0 && k < kKernelKinds) ? names[k] : "";
}


namespace {

// Per-device launch facts of one geometry: the block-local kernel needs more
// than the 48 KB of shared memory a launch gets without opting in (the
// opt-in is per device), and persistent grids are sized from occupancy.
struct GeoLaunch {
    bool ready = false;
    int sms = 0;
    int occ_local = 0, occ_merge = 0, occ_write = 0;
};

template <class G>
bool geo_launch(GeoLaunch &out) {
    static std::mutex mu;
    static GeoLaunch per_dev[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return false;
    std::lock_guard<std::mutex> lk(mu);
    GeoLaunch &g = per_dev[dev];
    if (!g.ready) {
        const int bytes = (int)sizeof(LocalSmem<G>);
        if (cudaFuncSetAttribute(k_block_local<G, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) !=
                cudaSuccess ||
            cudaFuncSetAttribute(k_block_local<G, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) !=
                cudaSuccess)
            return false;
        if (cudaDeviceGetAttribute(&g.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return false;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g.occ_local, k_block_local<G, true>, G::kThreads,
                                                          bytes) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g.occ_merge, k_block_merge<G, true>, G::kBW, 0) !=
                cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g.occ_write, k_block_write<G>, G::kThreads, 0) !=
                cudaSuccess)
            return false;
        g.occ_local = std::max(1, g.occ_local);
        g.occ_merge = std::max(1, g.occ_merge);
        g.occ_write = std::max(1, g.occ_write);
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
    local_cap = cap > 0 ? cap : kLabCap * G::kThreads + 16;
    global_cap = cap > 0 ? cap : (int)(slots + 16 < (1LL << 30) ? slots + 16 : (1LL << 30));
    bound = (uint32_t)slots;
}

template <class G>
int launch_table(int conn, const JobTable &jt, unsigned grid_local, unsigned grid_merge, unsigned grid_write,
                 const Scratch &s, int local_cap, int global_cap, uint32_t bound, cudaStream_t stream) {
    cudaEvent_t ev = timing_mark(stream, nullptr, -1);
    if (conn == 8) {
        k_block_local<G, true><<<grid_local, G::kThreads, sizeof(LocalSmem<G>), stream>>>(jt, s, local_cap);
        ev = timing_mark(stream, ev, kKindLocal);
        k_block_merge<G, true><<<grid_merge, G::kBW, 0, stream>>>(jt, s, global_cap, bound);
    } else {
        k_block_local<G, false><<<grid_local, G::kThreads, sizeof(LocalSmem<G>), stream>>>(jt, s, local_cap);
        ev = timing_mark(stream, ev, kKindLocal);
        k_block_merge<G, false><<<grid_merge, G::kBW, 0, stream>>>(jt, s, global_cap, bound);
    }
    ev = timing_mark(stream, ev, kKindMerge);
    k_block_write<G><<<grid_write, G::kThreads, 0, stream>>>(jt, s, global_cap, bound);
    ev = timing_mark(stream, ev, kKindRelabel);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

template <class G>
int launch_single(const uint8_t *img, int H, int W, size_t pitch, int conn, int32_t *labels, void *ws,
                  cudaStream_t stream, int cap) {
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
    jt.single.flags = ((((uintptr_t)img | pitch) & 15) == 0 ? kJobVecIn : 0u) |
                      ((((uintptr_t)labels & 15) == 0 && (W & 3) == 0) ? kJobVecOut : 0u);
    const size_t nb = (size_t)jt.single.nbx * (size_t)jt.single.nby;
    jt.total = (unsigned)nb;
    int local_cap, global_cap;
    uint32_t bound;
    caps_for<G>(nb, cap, local_cap, global_cap, bound);
    return launch_table<G>(conn, jt, (unsigned)nb, (unsigned)nb, (unsigned)nb, carve<G>(ws, nb), local_cap,
                           global_cap, bound, stream);
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
    return launch_table<G>(conn, jt, (unsigned)(gl.sms * gl.occ_local), (unsigned)(gl.sms * gl.occ_merge),
                           (unsigned)(gl.sms * gl.occ_write), carve<G>(ws, capacity), local_cap, global_cap,
                           bound, stream);
}

}  // namespace

const char *geo_name(int geo) {
    static const char *names[kNumGeo] = {"512x64", "256x64", "1024x32"};
    return (geo >= 0 && geo < kNumGeo) ? names[geo] : "";
}

void geo_block_shape(int geo, int *bw, int *bh) {
    switch (geo) {
        case 1: *bw = G1::kBW; *bh = G1::kBH; break;
        case 2: *bw = G2::kBW; *bh = G2::kBH; break;
        default: *bw = G0::kBW; *bh = G0::kBH; break;
    }
}

size_t geo_blocks(int geo, int H, int W) {
    switch (geo) {
        case 1: return blocks_of<G1>(H, W);
        case 2: return blocks_of<G2>(H, W);
        default: return blocks_of<G0>(H, W);
    }
}

size_t geo_workspace_bytes(int geo, size_t blocks) {
    switch (geo) {
        case 1: return layout_for<G1>(blocks).total;
        case 2: return layout_for<G2>(blocks).total;
        default: return layout_for<G0>(blocks).total;
    }
}

size_t workspace_bytes(int H, int W) { return geo_workspace_bytes(0, geo_blocks(0, H, W)); }

int launch_label(const uint8_t *img, int H, int W, size_t pitch, int conn, int32_t *labels, void *ws,
                 cudaStream_t stream, int cap) {
    return launch_single<G0>(img, H, W, pitch, conn, labels, ws, stream, cap);
}

int prepare_geo(int geo) {
    GeoLaunch gl;
    switch (geo) {
        case 1: return geo_launch<G1>(gl) ? 0 : -1;
        case 2: return geo_launch<G2>(gl) ? 0 : -1;
        default: return geo_launch<G0>(gl) ? 0 : -1;
    }
}

int launch_jobs(int geo, int conn, JobHeader *hdr, const Job *jobs, void *ws, size_t capacity,
                cudaStream_t stream, int cap) {
    switch (geo) {
        case 1: return launch_batch<G1>(conn, hdr, jobs, ws, capacity, stream, cap);
        case 2: return launch_batch<G2>(conn, hdr, jobs, ws, capacity, stream, cap);
        default: return launch_batch<G0>(conn, hdr, jobs, ws, capacity, stream, cap);
    }
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
