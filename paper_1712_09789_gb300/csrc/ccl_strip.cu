// ccl_strip.cu -- strip sharding of one image: the boundary analysis of
// Sec. 3.2 applied at the seams between horizontal strips that are labelled
// separately (one strip per GPU, or several strips on one GPU).
//
// A strip is rows [y0, y0 + H) of an H_total x W image.  Its labelling runs
// in two halves around an exchange between the strips:
//   1. ccl_strip_begin: step 1 and the block merge on the strip alone, with
//      every key a raster position of the whole image (pixel (x, y) of the
//      strip is x + (y0 + y) * W).  Then k_strip_edges reads, for every
//      column of the strip's first and last row, the key of its component's
//      root within the strip (its smallest position there).
//   2. The callers gather the edge rows of all strips, in strip order.
//   3. ccl_strip_resolve (host): a union-find over the keys of the seam rows
//      joins every pair of foreground pixels adjacent across a seam (Eq. 1-2
//      at a strip edge) and lists each key whose component reaches a smaller
//      key through some seam, with that smallest key.
//   4. ccl_strip_finish: k_strip_rekey replaces the key of every root of the
//      strip that the list names, then the write-out runs as usual, so every
//      pixel gets 1 + the smallest position of its component in the whole
//      image.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/ccl.h"
#include "ccl_internal.h"

namespace {

constexpr int kStripErrCap = 1;
__device__ int g_strip_error = 0;

// Key of the root of union-find entry s (read-only walk with an iteration
// cap; 0xFFFFFFFF and the error bit when the walk is cut short).
__device__ __forceinline__ uint32_t strip_root_key(const uint64_t *P, uint32_t s, uint32_t bound, int cap,
                                                   int &err) {
    for (int i = 0; i < cap; ++i) {
        const uint64_t v = P[s];
        const uint32_t p = (uint32_t)v;
        if (p == s) return (uint32_t)(v >> 32);
        if (p >= bound) break;
        s = p;
    }
    err |= kStripErrCap;
    return 0xFFFFFFFFu;
}

// Edge rows of a strip: out[x] (first row) and out[W + x] (last row) = key of
// the pixel's root in the strip's merged union-find, 0xFFFFFFFF for
// background.  One thread per pixel of the two rows.
__global__ void k_strip_edges(ccl::ScratchView v, int W, uint32_t *out, int cap) {
    const unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 2u * (unsigned)W) return;
    const int row = (int)(i / (unsigned)W), x = (int)(i % (unsigned)W);
    const unsigned by = row ? v.nby - 1 : 0u;
    const unsigned b = by * v.nbx + (unsigned)(x / ccl::kStripBW);
    const uint16_t e =
        v.edges[(size_t)b * ccl::kStripEdge + (row ? ccl::kStripEdgeBottom : 0) + (x % ccl::kStripBW)];
    uint32_t key = 0xFFFFFFFFu;
    int err = 0;
    if (e != ccl::kStripNoSlot && e < ccl::kStripSlots) {
        const uint32_t bound = v.nbx * v.nby * (uint32_t)ccl::kStripSlots;
        key = strip_root_key(v.P, b * (uint32_t)ccl::kStripSlots + e, bound, cap, err);
    }
    out[i] = key;
    if (err) atomicOr(&g_strip_error, err);
}

// Every root entry of the strip's union-find whose key the sorted list
// `map` (pairs key, smallest key) names takes the smallest key.  One thread
// per entry; only roots are written, each by its own thread.
__global__ void k_strip_rekey(ccl::ScratchView v, const uint32_t *map, unsigned n) {
    const unsigned nb = v.nbx * v.nby;
    const unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nb * (unsigned)ccl::kStripSlots) return;
    const unsigned b = i / (unsigned)ccl::kStripSlots, k = i % (unsigned)ccl::kStripSlots;
    if ((int)k >= v.nslots[b]) return;
    const uint64_t e = v.P[i];
    if ((uint32_t)e != i) return;
    const uint32_t key = (uint32_t)(e >> 32);
    unsigned lo = 0, hi = n;
    while (lo < hi) {
        const unsigned mid = (lo + hi) >> 1;
        if (map[2 * mid] < key) lo = mid + 1;
        else hi = mid;
    }
    if (lo < n && map[2 * lo] == key) v.P[i] = ((uint64_t)map[2 * lo + 1] << 32) | (uint64_t)i;
}

// Argument rules shared by begin and finish.
ccl_status check_strip(int H, int W, int conn, int y0, int H_total, size_t ws_bytes, const void *ws) {
    if (H < 0 || W < 0 || y0 < 0 || H_total < 0 || (conn != 4 && conn != 8)) return CCL_ERR_INVALID_ARG;
    if ((long long)y0 + H > (long long)H_total) return CCL_ERR_INVALID_ARG;
    if ((long long)H_total * (long long)W > 2147483646LL) return CCL_ERR_UNSUPPORTED;
    // seams sit on block rows: a strip starts on a multiple of the block
    // height, and every strip but the last spans whole block rows
    if (y0 % ccl::kStripBH != 0) return CCL_ERR_INVALID_ARG;
    if (y0 + H != H_total && H % ccl::kStripBH != 0) return CCL_ERR_INVALID_ARG;
    if (H == 0 || W == 0) return CCL_OK;
    if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255) != 0 || ws_bytes < ccl::workspace_bytes(H, W))
        return CCL_ERR_INVALID_ARG;
    return CCL_OK;
}

int iteration_cap_default(int H, int W) {
    const long long slots = (((long long)W + ccl::kStripBW - 1) / ccl::kStripBW) *
                            (((long long)H + ccl::kStripBH - 1) / ccl::kStripBH) * ccl::kStripSlots;
    return (int)std::min<long long>(slots + 16, 1LL << 30);
}

}  // namespace

namespace ccl {

int read_and_clear_strip_error(int *value) {
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_strip_error, sizeof(int)) != cudaSuccess) return -1;
    if (v) {
        const int zero = 0;
        if (cudaMemcpyToSymbol(g_strip_error, &zero, sizeof(int)) != cudaSuccess) return -1;
    }
    *value = v;
    return 0;
}

}  // namespace ccl

extern "C" {

ccl_status ccl_strip_begin(const uint8_t *img, int H, int W, size_t pitch, int connectivity, int y0, int H_total,
                           void *workspace, size_t workspace_bytes, uint32_t *edges, void *stream) {
    ccl_status st = check_strip(H, W, connectivity, y0, H_total, workspace_bytes, workspace);
    if (st != CCL_OK || H == 0 || W == 0) return st;
    if (!img || !edges || pitch < (size_t)W) return CCL_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int cap = ccl::iteration_cap_api();
    // the write-out does not run here: no labels are written yet
    if (ccl::launch_label_phases(img, H, W, pitch, connectivity, (uint32_t)y0 * (uint32_t)W, nullptr, workspace, s,
                                 cap, ccl::kPhaseLocalMerge) != 0)
        return CCL_ERR_CUDA;
    ccl::ScratchView v;
    ccl::label_scratch_view(H, W, connectivity, workspace, &v);
    const unsigned n = 2u * (unsigned)W;
    k_strip_edges<<<(n + 255) / 256, 256, 0, s>>>(v, W, edges, cap > 0 ? cap : iteration_cap_default(H, W));
    return cudaGetLastError() == cudaSuccess ? CCL_OK : CCL_ERR_CUDA;
}

ccl_status ccl_strip_resolve(const uint32_t *edges, int strips, int W, int connectivity, uint32_t *map,
                             size_t capacity, size_t *count) {
    if (!count || strips < 0 || W < 0 || (connectivity != 4 && connectivity != 8)) return CCL_ERR_INVALID_ARG;
    *count = 0;
    if (strips < 2 || W == 0) return CCL_OK;
    if (!edges) return CCL_ERR_INVALID_ARG;
    const size_t row = (size_t)W;
    const int seams = strips - 1;
    const uint32_t kEmpty = 0xFFFFFFFFu;
    const auto top = [&](int g) { return edges + (size_t)g * 2 * row; };
    const auto bottom = [&](int g) { return edges + (size_t)g * 2 * row + row; };
    // elements: the runs of the seam rows (consecutive foreground pixels of
    // one key: row neighbours are always one component)
    struct Run {
        int a, b;  // first and last column
        uint32_t key, el;
    };
    std::vector<uint32_t> parent;
    const auto find = [&](uint32_t x) {
        while (parent[x] != x) {
            parent[x] = parent[parent[x]];
            x = parent[x];
        }
        return x;
    };
    const auto unite = [&](uint32_t a, uint32_t b) {
        a = find(a);
        b = find(b);
        if (a != b) parent[a < b ? b : a] = a < b ? a : b;
    };
    // run starts and ends as bit masks (no branch per pixel: the rows of a
    // noisy image would mispredict on every other pixel), then one step per run
    const size_t words = (row + 63) / 64;
    std::vector<uint64_t> first(words), last(words);
    const auto runs_of = [&](const uint32_t *r, std::vector<Run> &out) {
        out.clear();
        for (size_t w = 0; w < words; ++w) {
            uint64_t f = 0, l = 0;
            const size_t x0 = w * 64, x1 = std::min(row, x0 + 64);
            for (size_t x = x0; x < x1; ++x) {
                const uint32_t k = r[x];
                const uint32_t kp = x > 0 ? r[x - 1] : kEmpty;
                const uint32_t kn = x + 1 < row ? r[x + 1] : kEmpty;
                f |= (uint64_t)(k != kEmpty && k != kp) << (x - x0);
                l |= (uint64_t)(k != kEmpty && k != kn) << (x - x0);
            }
            first[w] = f;
            last[w] = l;
        }
        size_t wl = 0;
        uint64_t lbits = last[0];
        for (size_t w = 0; w < words; ++w)
            for (uint64_t f = first[w]; f; f &= f - 1) {
                const int a = (int)(w * 64) + __builtin_ctzll(f);
                // the run's last column: the first end at or after its start
                while (!lbits) lbits = last[++wl];
                const int b = (int)(wl * 64) + __builtin_ctzll(lbits);
                lbits &= lbits - 1;
                out.push_back({a, b, r[a], (uint32_t)parent.size()});
                parent.push_back((uint32_t)parent.size());
            }
    };
    // per row, key -> first run holding it (open addressing, 2W..4W slots);
    // the first row of strip g stays available while its last row is read
    size_t cap = 16;
    int cap_log2 = 4;
    while (cap < 2 * row) {
        cap <<= 1;
        ++cap_log2;
    }
    std::vector<uint32_t> hk[2] = {std::vector<uint32_t>(cap), std::vector<uint32_t>(cap)};
    std::vector<uint32_t> hv[2] = {std::vector<uint32_t>(cap), std::vector<uint32_t>(cap)};
    std::vector<uint32_t> bk(cap), bv(cap);
    const auto slot_of = [&](const std::vector<uint32_t> &k, uint32_t key) {
        // Fibonacci hashing: the top bits of the product mix every bit of
        // the key (keys of one row often share their low bits)
        size_t h = (size_t)(((uint64_t)key * 0x9E3779B97F4A7C15ull) >> (64 - cap_log2));
        while (k[h] != kEmpty && k[h] != key) h = (h + 1) & (cap - 1);
        return h;
    };
    // every distinct key once, with one element that holds it
    std::vector<std::pair<uint32_t, uint32_t>> distinct;
    std::vector<Run> ur, dr;
    const int reach = connectivity == 8 ? 1 : 0;
    bool have_top = false;  // table (s & 1) ^ 1 holds the first row of strip s
    for (int s = 0; s < seams; ++s) {
        // the last row of strip s: equal keys are one component; a key that
        // also sits on the first row of strip s is that row's component
        runs_of(bottom(s), ur);
        std::fill(bk.begin(), bk.end(), kEmpty);
        const std::vector<uint32_t> &tk = hk[(s & 1) ^ 1], &tv = hv[(s & 1) ^ 1];
        for (const Run &u : ur) {
            const size_t h = slot_of(bk, u.key);
            if (bk[h] == u.key) {
                unite(u.el, bv[h]);
                continue;
            }
            bk[h] = u.key;
            bv[h] = u.el;
            const size_t ht = have_top ? slot_of(tk, u.key) : 0;
            if (have_top && tk[ht] == u.key) unite(u.el, tv[ht]);
            else distinct.emplace_back(u.key, u.el);
        }
        // the first row of strip s + 1
        runs_of(top(s + 1), dr);
        std::vector<uint32_t> &nk = hk[s & 1], &nv = hv[s & 1];
        std::fill(nk.begin(), nk.end(), kEmpty);
        for (const Run &d : dr) {
            const size_t h = slot_of(nk, d.key);
            if (nk[h] == d.key) {
                unite(d.el, nv[h]);
                continue;
            }
            nk[h] = d.key;
            nv[h] = d.el;
            distinct.emplace_back(d.key, d.el);
        }
        have_top = true;
        // runs that touch across the seam: column ranges that overlap, each
        // upper run widened by one column on both sides under 8-connectivity.
        // Widened upper runs may share a column with their neighbour, so on
        // equal ends the upper run moves on: the next lower run starts two
        // columns further at least and cannot touch it.
        size_t i = 0, k = 0;
        while (i < ur.size() && k < dr.size()) {
            const Run &u = ur[i], &d = dr[k];
            if (d.a <= u.b + reach && u.a - reach <= d.b) unite(u.el, d.el);
            if (u.b + reach <= d.b) ++i;
            else ++k;
        }
    }
    // smallest key of every set, then the keys that change
    std::vector<uint32_t> least(parent.size(), kEmpty);
    for (const auto &d : distinct) {
        uint32_t &m = least[find(d.second)];
        m = std::min(m, d.first);
    }
    std::vector<std::pair<uint32_t, uint32_t>> out;
    for (const auto &d : distinct) {
        const uint32_t m = least[find(d.second)];
        if (m < d.first) out.emplace_back(d.first, m);
    }
    std::sort(out.begin(), out.end());
    const size_t n = out.size();
    if (map)
        for (size_t i = 0; i < n && i < capacity; ++i) {
            map[2 * i] = out[i].first;
            map[2 * i + 1] = out[i].second;
        }
    *count = n;
    return (n > capacity || (n && !map)) ? CCL_ERR_INVALID_ARG : CCL_OK;
}

ccl_status ccl_strip_finish(int H, int W, int connectivity, int y0, int H_total, const uint32_t *map, size_t count,
                            int32_t *labels, void *workspace, size_t workspace_bytes, void *stream) {
    ccl_status st = check_strip(H, W, connectivity, y0, H_total, workspace_bytes, workspace);
    if (st != CCL_OK || H == 0 || W == 0) return st;
    if (!labels || (count && !map) || count > 0xFFFFFFFFull) return CCL_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    ccl::ScratchView v;
    ccl::label_scratch_view(H, W, connectivity, workspace, &v);
    if (count) {
        const unsigned n = v.nbx * v.nby * (unsigned)ccl::kStripSlots;
        k_strip_rekey<<<(n + 255) / 256, 256, 0, s>>>(v, map, (unsigned)count);
        if (cudaGetLastError() != cudaSuccess) return CCL_ERR_CUDA;
    }
    // the write-out reads only the scratch (masks, values, border records,
    // union-find): the image is not needed again
    if (ccl::launch_label_phases(nullptr, H, W, (size_t)W, connectivity, (uint32_t)y0 * (uint32_t)W, labels,
                                 workspace, s, ccl::iteration_cap_api(), ccl::kPhaseWrite) != 0)
        return CCL_ERR_CUDA;
    return CCL_OK;
}

}  // extern "C"
