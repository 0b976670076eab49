// ccl_kernels.cu -- the three steps of the block-based labeller as sm_103a
// kernels, and the launcher that enqueues them on a stream.
//
//   k_block_local   step 1, Kernel 1 (Sec. 3.1) on 512 x 64 blocks: every
//                   thread labels its 32 x 8 lane tile by coarse labelling
//                   (row connection by bit operations; column connection to
//                   the first run above; unification through the list) and
//                   refinement (merging the further runs above); the lane
//                   tiles of the block are then merged along their seams.
//                   Writes the block's row masks, one value per run (block key
//                   of its root, or its border slot), the border record of
//                   the block and one global union-find entry per border
//                   component.
//   k_block_merge   step 2, Kernel 2 (Sec. 3.2, Eq. 1-2): only the pixel
//                   pairs that straddle a block edge are examined.
//   k_block_write   step 3 (Sec. 3.3): root-find for the block's border slots
//                   in the merged union-find, then expands the per-run values
//                   over the row masks and writes every label once.
//
// HBM traffic per pixel: 1 B image read, 4 B label write, plus the row masks
// (1/8 B written, 1/8 B read) and the per-run values (1 B label and 2 B value
// per run, written and read once), most of which stay in L2.
#include <cstdint>
#include <deque>
#include <mutex>
#include <vector>

#include <cuda_runtime.h>

#include "ccl_block.cuh"
#include "ccl_internal.h"

namespace ccl {

__device__ int g_device_error = 0;

struct ImageArgs {
    const uint8_t *img;
    int32_t *labels;
    size_t pitch;
    int H, W;
    int nbx, nby;
    bool vec_ok;       // img and pitch 16-byte aligned
    bool out_vec_ok;   // labels 16-byte aligned and W % 4 == 0
};

// Per-block scratch regions (all sized for capacity; only used parts are
// touched).
struct Scratch {
    uint32_t *masks;   // [blocks][128 lane tiles][8 rows]
    uint32_t *lstream; // [blocks][kLWords][128]: run labels, 4 per word
    uint4 *vstream;    // [blocks][kVChunks][128]: run values, 8 per chunk
    uint16_t *edges;   // [blocks][kEdge]
    uint64_t *P;       // [blocks][kSlots]
    int32_t *nslots;   // [blocks]
};

__device__ __forceinline__ void report(int err) {
    if (err) atomicOr(&g_device_error, err);
}

// ---------------------------------------------------------------------------
struct LocalSmem {
    uint16_t par[kLabCap * kThreads];            // list entries, see ccl_block.cuh
    uint8_t lab[3][kLW][kLabPitch];              // run-start labels: row 0, then two alternating rows
    uint8_t lcol[kLH][kLabPitch];                // label of the run holding column 0, per row
    uint8_t rcol[kLH][kLabPitch];                // label of the run holding column 31, per row
    uint32_t mask[kLH][kThreads];                // row masks
    union {
        uint16_t qpair[16][kThreads];            // further contacts of the current row (scan)
        struct {
            uint32_t border[kLabCap * kThreads / 32];  // bit per id: root touching the block border
            uint32_t prefix[kLabCap * kThreads / 32];
        };
    };
    uint32_t warp_tot[kThreads / 32];
    int nslots;
    int err;
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

template <bool kConn8>
__global__ void __launch_bounds__(kThreads, 4) k_block_local(ImageArgs a, Scratch s, int cap) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    LocalSmem &sm = *reinterpret_cast<LocalSmem *>(smem_raw);
    const int b = blockIdx.x;
    const int bx = b % a.nbx, by = b / a.nbx;
    const int x0 = bx * kBW, y0 = by * kBH;
    const int t = threadIdx.x;
    const int tx = t & (kBLX - 1), ty = t >> 4;
    const int xl = x0 + kLW * tx, yl = y0 + kLH * ty;
    int err = 0;

    if (t == 0) sm.err = 0;

    // -- initialization: the lane tile's 8 rows as masks (all loads in flight
    // at once; pixels outside the image are background)
    uint32_t mrow[kLH];
    if (a.vec_ok && xl + kLW <= a.W && yl + kLH <= a.H) {
        uint4 raw[2 * kLH];
        const uint8_t *p = a.img + (size_t)yl * a.pitch + xl;
#pragma unroll
        for (int r = 0; r < kLH; ++r) {
            raw[2 * r] = ldg_nc16(p + (size_t)r * a.pitch);
            raw[2 * r + 1] = ldg_nc16(p + (size_t)r * a.pitch + 16);
        }
#pragma unroll
        for (int r = 0; r < kLH; ++r) mrow[r] = nz16(raw[2 * r]) | (nz16(raw[2 * r + 1]) << 16);
    } else {
#pragma unroll
        for (int r = 0; r < kLH; ++r) {
            uint32_t m = 0;
            const int y = yl + r;
            if (y < a.H && xl < a.W) {
                const uint8_t *p = a.img + (size_t)y * a.pitch + xl;
                const int n = a.W - xl < kLW ? a.W - xl : kLW;
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
    uint32_t *lout = s.lstream + (size_t)b * kLWords * kThreads + t;
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
            if (P) L = prev[hibit(prevS & upto(u0)) * kLabPitch];
            else if (act) {
                vpar[nlab * kThreads + t] = (uint16_t)(kRoot | (r * kLW + a0));
                ++nlab;
            }
            uint32_t Q = P ? (prevS & P & ~upto(u0)) : 0u;
            while (__any_sync(kFull, Q != 0u)) {
                if (Q) {
                    sm.qpair[nq][t] = (uint16_t)(L | (prev[lobit(Q) * kLabPitch] << 8));
                    ++nq;
                    Q &= Q - 1u;
                }
            }
            if (act) {
                cur[a0 * kLabPitch] = (uint8_t)L;
                lacc = (lacc >> 8) | ((uint32_t)L << 24);
                ++nrun;
                if ((nrun & 3) == 0) lout[(size_t)((nrun >> 2) - 1) * kThreads] = lacc;
            }
        }
        sm.lcol[r][t] = (m & 1u) ? cur[0] : (uint8_t)0xFF;
        sm.rcol[r][t] = (m >> 31) ? cur[hibit(m & ~(m << 1)) * kLabPitch] : (uint8_t)0xFF;
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
                    const uint16_t e = vpar[A * kThreads + t];
                    if (e & kRoot) {
                        pa = false;
                    } else {
                        const int p = e & (kLabCap - 1);
                        const uint16_t g = vpar[p * kThreads + t];
                        if (g & kRoot) { A = p; pa = false; }
                        else { vpar[A * kThreads + t] = g; A = g & (kLabCap - 1); }
                    }
                }
                if (pb) {
                    const uint16_t e = vpar[B * kThreads + t];
                    if (e & kRoot) {
                        pb = false;
                    } else {
                        const int p = e & (kLabCap - 1);
                        const uint16_t g = vpar[p * kThreads + t];
                        if (g & kRoot) { B = p; pb = false; }
                        else { vpar[B * kThreads + t] = g; B = g & (kLabCap - 1); }
                    }
                }
                if (i >= cap) {
                    if (pa || pb) err |= kErrLocalCap;
                    break;
                }
            }
            if (hq && A != B) {
                const int lo = A < B ? A : B, hi = A < B ? B : A;
                vpar[hi * kThreads + t] = (uint16_t)lo;
            }
        }
        __syncwarp();
    }
    if (nrun & 3) lout[(size_t)(nrun >> 2) * kThreads] = lacc >> (8 * (4 - (nrun & 3)));
    // compress the own lists (labels are still lane-local here, so no other
    // lane reads them) and turn parent links into block-wide ids: the thread
    // index joins the label
    const int nlab_max = __reduce_max_sync(kFull, nlab);
    for (int L = 0; L < nlab_max; ++L) {
        if (L < nlab) {
            // entries already converted by earlier rounds carry this thread's
            // index in their high bits; the low bits are the lane-local label
            int x = L;
            uint16_t e = vpar[x * kThreads + t];
            for (int i = 0; !(e & kRoot) && i < cap; ++i) {
                x = e & (kLabCap - 1);
                e = vpar[x * kThreads + t];
            }
            if (x != L) vpar[L * kThreads + t] = (uint16_t)((t << 7) | x);
        }
    }
    __syncthreads();

    // the refinement queue is dead now; its space holds the border bitmap
    for (int i = t; i < kLabCap * kThreads / 32; i += kThreads) sm.border[i] = 0u;

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
            union_block_sync(sm.par, me_fg && at_l && !(up_me && up_l), me, (tl << 7) | sm.rcol[r][tl], cap, err);
            if (kConn8) {
                union_block_sync(sm.par, me_fg && up_l && !up_me, me,
                                 (tl << 7) | sm.rcol[r > 0 ? r - 1 : 0][tl], cap, err);
                union_block_sync(sm.par, me_fg && dn_l && !dn_me, me,
                                 (tl << 7) | sm.rcol[r + 1 < kLH ? r + 1 : r][tl], cap, err);
            }
        }
    }
    {
        const bool hasu = ty > 0;
        const int tu = hasu ? t - kBLX : t;
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
            const int me = (t << 7) | top[a0 * kLabPitch];
            const int u0 = P ? lobit(P) : 0;
            union_block_sync(sm.par, P != 0u, me, (tu << 7) | bot[hibit((SU & upto(u0)) | 1u) * kLabPitch], cap,
                             err);
            uint32_t Q = P ? (SU & P & ~upto(u0)) : 0u;
            while (__any_sync(kFull, Q != 0u)) {
                const bool hq = Q != 0u;
                const int q = hq ? lobit(Q) : 0;
                Q &= Q - 1u;
                union_block_sync(sm.par, hq, me, (tu << 7) | bot[q * kLabPitch], cap, err);
            }
        }
        if (kConn8) {
            // corners: the lane tiles up-left and up-right
            const bool ul = hasu && tx > 0 && (m0 & 1u);
            const int tul = ul ? tu - 1 : t;
            const uint32_t mUL = ul ? sm.mask[kLH - 1][tul] : 0u;
            const uint32_t SUL = mUL & ~(mUL << 1);
            union_block_sync(sm.par, ul && (mUL >> 31), (t << 7) | top[0],
                             (tul << 7) | sm.lab[lab_buf(kLH - 1)][hibit(SUL | 1u)][tul], cap, err);
            const bool ur = hasu && tx + 1 < kBLX && (m0 >> 31);
            const int tur = ur ? tu + 1 : t;
            const uint32_t S0 = m0 & ~(m0 << 1);
            union_block_sync(sm.par, ur && (sm.mask[kLH - 1][tur] & 1u), (t << 7) | top[hibit(S0 | 1u) * kLabPitch],
                             (tur << 7) | sm.lab[lab_buf(kLH - 1)][0][tur], cap, err);
        }
    }
    __syncthreads();

    // -- compress: every own list entry points straight at its root (the
    // finds only read, so every store here is a final root)
    for (int L = 0; L < nlab_max; ++L) {
        if (L < nlab) {
            const int id = (t << 7) | L;
            const int root = find_root_ro(vpar, id, cap, err);
            if (root != id) vpar[L * kThreads + t] = (uint16_t)root;
        }
    }
    __syncthreads();

    // -- roots that own a pixel of the block border
    auto root_of = [&](int id) -> int {
        const uint16_t e = vpar[par_index(id)];
        return (e & kRoot) ? id : (int)e;
    };
    auto mark = [&](int id) {
        const int root = root_of(id);
        atomicOr(&sm.border[root >> 5], 1u << (root & 31));
    };
    if (ty == 0)
        for (uint32_t S = m0 & ~(m0 << 1); S; S &= S - 1) mark((t << 7) | sm.lab[0][lobit(S)][t]);
    if (ty == kBLY - 1) {
        const uint32_t m7 = mrow[kLH - 1];
        for (uint32_t S = m7 & ~(m7 << 1); S; S &= S - 1)
            mark((t << 7) | sm.lab[lab_buf(kLH - 1)][lobit(S)][t]);
    }
    if (tx == 0) {
#pragma unroll
        for (int r = 0; r < kLH; ++r)
            if (mrow[r] & 1u) mark((t << 7) | sm.lcol[r][t]);
    }
    if (tx == kBLX - 1) {
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
        // at most kSlots border components exist; more marks only after an
        // iteration cap was hit, and the surplus slots are dropped
        if (t == kThreads - 1) {
            sm.nslots = (int)(base + incl) < kSlots ? (int)(base + incl) : kSlots;
            if ((int)(base + incl) > kSlots) sm.err |= kErrLocalCap;
        }
    }
    __syncthreads();
    auto slot_of = [&](int root) -> int {
        return (int)(sm.prefix[root >> 5] + __popc(sm.border[root >> 5] & ((1u << (root & 31)) - 1u)));
    };

    // -- one global union-find entry per border component, keyed by its
    // minimum global raster position (ID conversion, Sec. 3.1.4)
    {
        const uint32_t sbase = (uint32_t)b * kSlots;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int word = 4 * t + k;
            uint32_t bits = sm.border[word];
            uint32_t slot = sm.prefix[word];
            for (; bits && slot < (uint32_t)kSlots; bits &= bits - 1, ++slot) {
                const int root = word * 32 + lobit(bits);
                const int key = root_key(root, vpar[par_index(root)]);
                const uint32_t g = (uint32_t)(y0 + (key >> kBWLog2)) * (uint32_t)a.W +
                                   (uint32_t)(x0 + (key & (kBW - 1)));
                s.P[sbase + slot] = pack_slot(g, sbase + slot);
            }
        }
    }
    __syncthreads();
    // -- each own root entry becomes the value its runs carry from now on
    for (int L = 0; L < nlab_max; ++L) {
        if (L < nlab) {
            const int id = (t << 7) | L;
            const uint16_t e = vpar[L * kThreads + t];
            if (e & kRoot) {
                const bool border = (sm.border[id >> 5] >> (id & 31)) & 1u;
                vpar[L * kThreads + t] = border ? (uint16_t)(kRootBorder | slot_of(id))
                                                : (uint16_t)(kRoot | root_key(id, e));
            }
        }
    }
    __syncthreads();
    // ... and so does every own non-root entry (it points straight at a root,
    // whose value is final), making a run's value a single lookup
    for (int L = 0; L < nlab_max; ++L) {
        if (L < nlab) {
            const uint16_t e = vpar[L * kThreads + t];
            if (e < kRootBorder) vpar[L * kThreads + t] = vpar[par_index(e)];
        }
    }

    // -- border record of the block: the slot of every border pixel
    uint16_t *Eb = s.edges + (size_t)b * kEdge;
    if (ty == 0 || ty == kBLY - 1) {
        const int rr = ty == 0 ? 0 : kLH - 1;
        const uint32_t m = mrow[rr];
        const uint32_t S = m & ~(m << 1);
        const uint8_t *lb = &sm.lab[lab_buf(rr)][0][t];
        uint16_t *dst = Eb + (ty == 0 ? kEdgeTop : kEdgeBottom) + kLW * tx;
#pragma unroll 4
        for (int c = 0; c < kLW; ++c) {
            uint16_t v = kBg;
            if ((m >> c) & 1u) v = border_slot(run_value(vpar, (t << 7) | lb[hibit(S & upto(c)) * kLabPitch]));
            dst[c] = v;
        }
    }
    if (tx == 0 || tx == kBLX - 1) {
        uint16_t *dst = Eb + (tx == 0 ? kEdgeLeft : kEdgeRight) + kLH * ty;
#pragma unroll
        for (int r = 0; r < kLH; ++r) {
            const bool fg = tx == 0 ? (mrow[r] & 1u) : (mrow[r] >> 31);
            const int L = tx == 0 ? sm.lcol[r][t] : sm.rcol[r][t];
            dst[r] = fg ? border_slot(run_value(vpar, (t << 7) | L)) : kBg;
        }
    }
    // -- per-run values: block key of the root, or kBorderFlag | slot
    {
        const uint32_t *lin = s.lstream + (size_t)b * kLWords * kThreads + t;
        uint4 *vout = s.vstream + (size_t)b * kVChunks * kThreads + t;
        HalfQueue vq;
        const int nrun_max = __reduce_max_sync(kFull, nrun);
        for (int k = 0; k < nrun_max; k += 4) {
            const uint32_t w = k < nrun ? lin[(size_t)(k >> 2) * kThreads] : 0u;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (k + j < nrun) {
                    vq.push(run_value(vpar, (t << 7) | ((w >> (8 * j)) & 0xFF)));
                    if (((k + j + 1) & 7) == 0) vout[(size_t)((k + j) >> 3) * kThreads] = vq.bits();
                }
            }
        }
        if (nrun & 7) {
            for (int k = nrun & 7; k < 8; ++k) vq.push(0);
            vout[(size_t)(nrun >> 3) * kThreads] = vq.bits();
        }
    }
    // -- row masks for the write-out pass
    {
        uint4 *mo = reinterpret_cast<uint4 *>(s.masks + ((size_t)b * kThreads + t) * kLH);
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

// ---------------------------------------------------------------------------
// Each block examines the pixel pairs across its top edge, its left edge and
// (8-connectivity) its two upper corners; the right, bottom and lower corners
// belong to the neighbouring blocks.  A pair that repeats the pair of the
// neighbouring pixel is skipped.
constexpr int kMergeThreads = kBW;  // one thread per top-edge column

template <bool kConn8>
__global__ void __launch_bounds__(kMergeThreads) k_block_merge(Scratch s, int nbx, int nby, int cap) {
    const int b = blockIdx.x;
    const int bx = b % nbx, by = b / nbx;
    const uint16_t *E = s.edges + (size_t)b * kEdge;
    const uint32_t base = (uint32_t)b * kSlots;
    const uint32_t bound = (uint32_t)nbx * (uint32_t)nby * kSlots;
    int err = 0;
    // every slot named by a border record is below its block's slot count;
    // checking it keeps the finds inside initialised entries whatever happened
    const auto valid = [&](int blk, uint16_t v) { return v != kBg && (int)v < s.nslots[blk]; };

    if (by > 0) {
        const int bu = b - nbx;
        const uint16_t *Eu = s.edges + (size_t)bu * kEdge;
        const uint32_t ubase = (uint32_t)bu * kSlots;
        for (int j = threadIdx.x; j < kBW; j += kMergeThreads) {
            const uint16_t a = E[kEdgeTop + j];
            if (!valid(b, a)) continue;
            const uint16_t aL = j > 0 ? E[kEdgeTop + j - 1] : kBg;
            const uint16_t aR = j + 1 < kBW ? E[kEdgeTop + j + 1] : kBg;
            const uint16_t c = Eu[kEdgeBottom + j];
            const uint16_t cL = j > 0 ? Eu[kEdgeBottom + j - 1] : kBg;
            if (valid(bu, c) && !(aL == a && cL == c)) union_global(s.P, base + a, ubase + c, cap, err, bound);
            if (kConn8) {
                if (j > 0) {
                    if (valid(bu, cL) && aL != a) union_global(s.P, base + a, ubase + cL, cap, err, bound);
                } else if (bx > 0) {
                    const uint16_t d = s.edges[(size_t)(bu - 1) * kEdge + kEdgeBottom + kBW - 1];
                    if (valid(bu - 1, d)) union_global(s.P, base + a, (uint32_t)(bu - 1) * kSlots + d, cap, err, bound);
                }
                if (j + 1 < kBW) {
                    const uint16_t cR = Eu[kEdgeBottom + j + 1];
                    if (valid(bu, cR) && aR != a) union_global(s.P, base + a, ubase + cR, cap, err, bound);
                } else if (bx + 1 < nbx) {
                    const uint16_t d = s.edges[(size_t)(bu + 1) * kEdge + kEdgeBottom + 0];
                    if (valid(bu + 1, d)) union_global(s.P, base + a, (uint32_t)(bu + 1) * kSlots + d, cap, err, bound);
                }
            }
        }
    }
    if (bx > 0) {
        const int bl = b - 1;
        const uint16_t *El = s.edges + (size_t)bl * kEdge;
        const uint32_t lbase = (uint32_t)bl * kSlots;
        for (int j = threadIdx.x; j < kBH; j += kMergeThreads) {
            const uint16_t a = E[kEdgeLeft + j];
            if (!valid(b, a)) continue;
            const uint16_t aU = j > 0 ? E[kEdgeLeft + j - 1] : kBg;
            const uint16_t aD = j + 1 < kBH ? E[kEdgeLeft + j + 1] : kBg;
            const uint16_t c = El[kEdgeRight + j];
            const uint16_t cU = j > 0 ? El[kEdgeRight + j - 1] : kBg;
            if (valid(bl, c) && !(aU == a && cU == c)) union_global(s.P, base + a, lbase + c, cap, err, bound);
            if (kConn8) {
                if (j > 0 && valid(bl, cU) && aU != a) union_global(s.P, base + a, lbase + cU, cap, err, bound);
                if (j + 1 < kBH) {
                    const uint16_t cD = El[kEdgeRight + j + 1];
                    if (valid(bl, cD) && aD != a) union_global(s.P, base + a, lbase + cD, cap, err, bound);
                }
            }
        }
    }
    report(err);
}

struct WriteSmem {
    int slot_label[kSlots];
    int runlab[kBLY][kBW];          // label of every run at its start column, one row of all lane tiles
    uint32_t mask[kLH][kThreads];   // row masks of the block
};

// Position of (lane tile tx, column c) in a runlab row: the column is XORed
// with tx so that the four lane tiles read by one warp of the copy-out spread
// over the banks.
__device__ __forceinline__ int runlab_index(int tx, int c) { return kLW * tx + (c ^ ((tx & 3) << 3)); }

__global__ void __launch_bounds__(kThreads, 4) k_block_write(ImageArgs a, Scratch s, int cap, uint32_t bound) {
    __shared__ WriteSmem sm;
    const int b = blockIdx.x;
    const int bx = b % a.nbx, by = b / a.nbx;
    const int x0 = bx * kBW, y0 = by * kBH;
    const int t = threadIdx.x;
    const int tx = t & (kBLX - 1), ty = t >> 4;

    // final label of each border slot: root-find in the merged union-find
    // (read-only; every union is complete when this kernel starts)
    const int ns = s.nslots[b];
    int err = 0;
    for (int k = t; k < ns; k += kThreads) {
        uint32_t key;
        find_global_ro(s.P, (uint32_t)b * kSlots + (uint32_t)k, key, cap, err, bound);
        sm.slot_label[k] = (int)key + 1;
    }
    report(err);

    const uint4 *mi = reinterpret_cast<const uint4 *>(s.masks + ((size_t)b * kThreads + t) * kLH);
    const uint4 mA = mi[0], mB = mi[1];
    const uint32_t mrow[kLH] = {mA.x, mA.y, mA.z, mA.w, mB.x, mB.y, mB.z, mB.w};
#pragma unroll
    for (int r = 0; r < kLH; ++r) sm.mask[r][t] = mrow[r];
    // per-run values, 8 per chunk; the next chunk is always already in flight
    const uint4 *vin = s.vstream + (size_t)b * kVChunks * kThreads + t;
    int nrun = 0;
#pragma unroll
    for (int r = 0; r < kLH; ++r) nrun += __popc(mrow[r] & ~(mrow[r] << 1));
    const int nchunks = (nrun + 7) >> 3;
    uint4 vq = nchunks > 0 ? vin[0] : make_uint4(0, 0, 0, 0);
    uint4 vnext = nchunks > 1 ? vin[kThreads] : make_uint4(0, 0, 0, 0);
    int vi = 0, vc = 2;
    __syncthreads();

    // copy-out geometry: thread t covers 4 pixels of every staged row
    const int q = t;                       // 4-pixel chunk of a 512-pixel row
    const int ctx = q >> 3;                // its lane tile
    const int c0 = (q & 7) * 4;            // its first column inside the lane tile
    const int x = x0 + 4 * q;

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
                    if (vc < nchunks) vnext = vin[(size_t)vc * kThreads];
                    ++vc;
                    vi = 0;
                }
                const uint32_t w = vi < 2 ? vq.x : vi < 4 ? vq.y : vi < 6 ? vq.z : vq.w;
                const uint32_t v = (w >> ((vi & 1) * 16)) & 0xFFFFu;
                ++vi;
                const uint32_t slot = v & 0x7FFFu;
                const int lab = (v & kBorderFlag) ? ((int)slot < ns ? sm.slot_label[slot] : 0)
                                                   : (int)((uint32_t)(y0 + (int)(v >> kBWLog2)) * (uint32_t)a.W +
                                                           (uint32_t)(x0 + (int)(v & (kBW - 1)))) + 1;
                sm.runlab[ty][runlab_index(tx, a0)] = lab;
            }
        }
        __syncthreads();
        // coalesced write-out of image rows y0 + 8*ry + r: every pixel takes
        // the label stored at the start of its run
#pragma unroll
        for (int ry = 0; ry < kBLY; ++ry) {
            const int y = y0 + kLH * ry + r;
            if (y < a.H && x < a.W) {
                const uint32_t mm = sm.mask[r][ry * kBLX + ctx];
                const uint32_t SS = mm & ~(mm << 1);
                int v[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int c = c0 + j;
                    v[j] = ((mm >> c) & 1u) ? sm.runlab[ry][runlab_index(ctx, hibit(SS & upto(c)))] : 0;
                }
                int32_t *dst = a.labels + (size_t)y * a.W + x;
                if (a.out_vec_ok && x + 4 <= a.W) {
                    __stcs(reinterpret_cast<int4 *>(dst), make_int4(v[0], v[1], v[2], v[3]));
                } else {
                    __stcs(dst, v[0]);
                    if (x + 1 < a.W) __stcs(dst + 1, v[1]);
                    if (x + 2 < a.W) __stcs(dst + 2, v[2]);
                    if (x + 3 < a.W) __stcs(dst + 3, v[3]);
                }
            }
        }
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

Layout layout_for(size_t nb) {
    Layout l;
    size_t off = 0;
    l.masks = off;   off += up256(nb * kThreads * kLH * sizeof(uint32_t));
    l.lstream = off; off += up256(nb * kLWords * kThreads * sizeof(uint32_t));
    l.vstream = off; off += up256(nb * kVChunks * kThreads * sizeof(uint4));
    l.edges = off;   off += up256(nb * kEdge * sizeof(uint16_t));
    l.P = off;       off += up256(nb * kSlots * sizeof(uint64_t));
    l.nslots = off;  off += up256(nb * sizeof(int32_t));
    l.total = off;
    return l;
}

size_t blocks_for(int H, int W) {
    return (((size_t)W + kBW - 1) / kBW) * (((size_t)H + kBH - 1) / kBH);
}

}  // namespace

size_t workspace_bytes(int H, int W) { return layout_for(blocks_for(H, W)).total; }

static Scratch carve(void *ws, int H, int W) {
    const Layout l = layout_for(blocks_for(H, W));
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
    static const char *names[kKernelKinds] = {"k_block_local", "k_block_merge", "k_block_write"};
    return (k >= 0 && k < kKernelKinds) ? names[k] : "";
}

// The block-local kernel needs more than the 48 KB of shared memory a launch
// gets without opting in; the opt-in is per device.
bool kernel_attributes_set() {
    static std::mutex mu;
    static bool done[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return false;
    std::lock_guard<std::mutex> lk(mu);
    if (done[dev]) return true;
    const int bytes = (int)sizeof(LocalSmem);
    if (cudaFuncSetAttribute(k_block_local<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) !=
            cudaSuccess ||
        cudaFuncSetAttribute(k_block_local<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) !=
            cudaSuccess)
        return false;
    done[dev] = true;
    return true;
}

int launch_label(const uint8_t *img, int H, int W, size_t pitch, int conn, int32_t *labels, void *ws,
                 cudaStream_t stream, int cap) {
    ImageArgs a;
    a.img = img;
    a.labels = labels;
    a.pitch = pitch;
    a.H = H;
    a.W = W;
    a.nbx = (W + kBW - 1) / kBW;
    a.nby = (H + kBH - 1) / kBH;
    a.vec_ok = ((reinterpret_cast<uintptr_t>(img) | pitch) & 15) == 0;
    a.out_vec_ok = (reinterpret_cast<uintptr_t>(labels) & 15) == 0 && (W & 3) == 0;
    const Scratch s = carve(ws, H, W);
    const unsigned nb = (unsigned)a.nbx * (unsigned)a.nby;
    // Default caps: a find walks a strictly decreasing chain, so it cannot
    // take more steps than there are list entries (slots); no valid input
    // reaches them.
    const long long slots = (long long)nb * kSlots + 16;
    const int local_cap = cap > 0 ? cap : kLabCap * kThreads + 16;
    const int global_cap = cap > 0 ? cap : (int)(slots < (1LL << 30) ? slots : (1LL << 30));
    if (!kernel_attributes_set()) return -1;
    cudaEvent_t ev = timing_mark(stream, nullptr, -1);
    if (conn == 8) {
        k_block_local<true><<<nb, kThreads, sizeof(LocalSmem), stream>>>(a, s, local_cap);
        ev = timing_mark(stream, ev, kKindLocal);
        k_block_merge<true><<<nb, kMergeThreads, 0, stream>>>(s, a.nbx, a.nby, global_cap);
    } else {
        k_block_local<false><<<nb, kThreads, sizeof(LocalSmem), stream>>>(a, s, local_cap);
        ev = timing_mark(stream, ev, kKindLocal);
        k_block_merge<false><<<nb, kMergeThreads, 0, stream>>>(s, a.nbx, a.nby, global_cap);
    }
    ev = timing_mark(stream, ev, kKindMerge);
    k_block_write<<<nb, kThreads, 0, stream>>>(a, s, global_cap, nb * (uint32_t)kSlots);
    ev = timing_mark(stream, ev, kKindRelabel);
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
