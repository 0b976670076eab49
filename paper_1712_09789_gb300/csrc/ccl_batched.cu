// ccl_batched.cu -- ccl_label_batched(): many images of uneven size labelled by
// one launch sequence of persistent kernels that take blocks from a device
// work queue, replayed as a CUDA graph, with the block shape picked by an
// autotuner.
//
// Per (device, stream, connectivity, block shape) the library keeps a runner:
// a device job table (header with the kernels' work counters, then one Job per
// image), the scratch for `capacity` blocks, and a ring of page-locked staging
// copies of the job table, each with its own instantiated graph.  A graph is
// [copy staging -> device table] + the labelling launches; a call fills the next
// ring slot (after the slot's previous replay has finished) and replays that
// slot's graph on the caller's stream.  Growing the capacity rebuilds the
// graphs.
//
// Autotuning: the block shapes are timed on a batch and the fastest is kept
// per (GPU name, connectivity, size class = log2 of the mean image area) in
// memory and in a text cache file ($CCL_AUTOTUNE_CACHE, else
// ~/.cache/ccl_gb300/autotune.txt).  $CCL_TILE (e.g. "256x64") overrides.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <string>
#include <sys/stat.h>
#include <tuple>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/ccl.h"
#include "ccl_internal.h"

namespace {

constexpr int kRing = 3;

struct Runner {
    int geo = 0, conn = 8, cap = 0;
    cudaStream_t capture = nullptr;
    unsigned char *d_table = nullptr;
    size_t cap_jobs = 0;
    void *d_ws = nullptr;
    size_t cap_blocks = 0;
    unsigned char *h_table[kRing] = {};
    cudaEvent_t done[kRing] = {};
    cudaGraphExec_t exec[kRing] = {};
    int next = 0;
};

std::mutex g_bmu;
std::map<std::tuple<int, cudaStream_t, int, int>, Runner *> g_runners;

size_t table_bytes(size_t jobs) { return sizeof(ccl::JobHeader) + jobs * sizeof(ccl::Job); }

void drop_graphs(Runner &R) {
    for (int i = 0; i < kRing; ++i) {
        if (R.done[i]) cudaEventSynchronize(R.done[i]);
        if (R.exec[i]) cudaGraphExecDestroy(R.exec[i]);
        R.exec[i] = nullptr;
    }
}

ccl_status ensure_capacity(Runner &R, size_t njobs, size_t blocks) {
    if (!R.capture && cudaStreamCreateWithFlags(&R.capture, cudaStreamNonBlocking) != cudaSuccess)
        return CCL_ERR_CUDA;
    for (int i = 0; i < kRing; ++i)
        if (!R.done[i] && cudaEventCreateWithFlags(&R.done[i], cudaEventDisableTiming) != cudaSuccess)
            return CCL_ERR_CUDA;
    if (njobs <= R.cap_jobs && blocks <= R.cap_blocks) return CCL_OK;
    drop_graphs(R);
    // doubling: a stream of growing batches (a server warming up) re-sizes,
    // re-allocates and re-captures only a few times
    const size_t nj = std::max(2 * njobs, std::max<size_t>(R.cap_jobs, 16));
    const size_t nb = std::max(2 * blocks, R.cap_blocks);
    if (R.d_table) cudaFree(R.d_table);
    if (R.d_ws) cudaFree(R.d_ws);
    R.d_table = nullptr;
    R.d_ws = nullptr;
    for (int i = 0; i < kRing; ++i) {
        if (R.h_table[i]) cudaFreeHost(R.h_table[i]);
        R.h_table[i] = nullptr;
    }
    R.cap_jobs = R.cap_blocks = 0;
    if (cudaMalloc(&R.d_table, table_bytes(nj)) != cudaSuccess ||
        cudaMalloc(&R.d_ws, ccl::geo_workspace_bytes(R.geo, nb)) != cudaSuccess) {
        cudaGetLastError();
        return CCL_ERR_OUT_OF_MEMORY;
    }
    for (int i = 0; i < kRing; ++i) {
        if (cudaMallocHost(&R.h_table[i], table_bytes(nj)) != cudaSuccess) {
            cudaGetLastError();
            return CCL_ERR_OUT_OF_MEMORY;
        }
        std::memset(R.h_table[i], 0, table_bytes(nj));
    }
    R.cap_jobs = nj;
    R.cap_blocks = nb;
    return CCL_OK;
}

ccl_status capture_slot(Runner &R, int slot) {
    if (ccl::prepare_geo(R.geo) != 0) return CCL_ERR_CUDA;
    if (cudaStreamBeginCapture(R.capture, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return CCL_ERR_CUDA;
    bool ok = cudaMemcpyAsync(R.d_table, R.h_table[slot], table_bytes(R.cap_jobs), cudaMemcpyHostToDevice,
                              R.capture) == cudaSuccess;
    ok = ok && ccl::launch_jobs(R.geo, R.conn, reinterpret_cast<ccl::JobHeader *>(R.d_table),
                                reinterpret_cast<const ccl::Job *>(R.d_table + sizeof(ccl::JobHeader)), R.d_ws,
                                R.cap_blocks, R.capture, R.cap) == 0;
    cudaGraph_t g = nullptr;
    const bool ended = cudaStreamEndCapture(R.capture, &g) == cudaSuccess;
    if (!ok || !ended || !g) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return CCL_ERR_CUDA;
    }
    const bool inst = cudaGraphInstantiate(&R.exec[slot], g, 0) == cudaSuccess;
    cudaGraphDestroy(g);
    if (!inst) {
        cudaGetLastError();
        R.exec[slot] = nullptr;
        return CCL_ERR_CUDA;
    }
    return CCL_OK;
}

struct Prepared {
    std::vector<ccl::Job> jobs;
    size_t blocks = 0;
};

ccl_status prepare(const ccl_image *images, int n, int conn, int geo, Prepared &out) {
    if (n < 0 || (n > 0 && !images) || (conn != 4 && conn != 8)) return CCL_ERR_INVALID_ARG;
    out.jobs.clear();
    out.blocks = 0;
    int bw = 0, bh = 0;
    ccl::geo_block_shape(geo, &bw, &bh);
    for (int i = 0; i < n; ++i) {
        const ccl_image &im = images[i];
        const ccl_status st = ccl::check_image_args_api(im.img, im.H, im.W, im.pitch, conn, im.labels);
        if (st != CCL_OK) return st;
        if (im.H == 0 || im.W == 0) continue;
        ccl::Job j;
        j.img = im.img;
        j.labels = im.labels;
        j.pitch = im.pitch;
        j.H = im.H;
        j.W = im.W;
        j.nbx = (im.W + bw - 1) / bw;
        j.nby = (im.H + bh - 1) / bh;
        j.block0 = (unsigned)out.blocks;
        j.key0 = 0;
        j.pad = 0;
        j.flags = ((((uintptr_t)im.img | im.pitch) & 15) == 0 ? ccl::kJobVecIn : 0u) |
                  ((((uintptr_t)im.labels & 15) == 0 && (im.W & 3) == 0) ? ccl::kJobVecOut : 0u);
        out.blocks += (size_t)j.nbx * (size_t)j.nby;
        if (out.blocks >= (size_t)1 << 31) return CCL_ERR_UNSUPPORTED;
        out.jobs.push_back(j);
    }
    return CCL_OK;
}

ccl_status run_batch(const Prepared &pb, int conn, int geo, cudaStream_t stream) {
    if (pb.jobs.empty()) return CCL_OK;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CCL_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_bmu);
    Runner *&rp = g_runners[std::make_tuple(dev, stream, conn, geo)];
    if (!rp) {
        rp = new Runner();
        rp->geo = geo;
        rp->conn = conn;
    }
    Runner &R = *rp;
    ccl_status st = ensure_capacity(R, pb.jobs.size(), pb.blocks);
    if (st != CCL_OK) return st;
    const int cap = ccl::iteration_cap_api();
    if (cap != R.cap) {
        drop_graphs(R);
        R.cap = cap;
    }
    const int slot = R.next;
    R.next = (R.next + 1) % kRing;
    if (cudaEventSynchronize(R.done[slot]) != cudaSuccess) return CCL_ERR_CUDA;
    ccl::JobHeader hdr{};
    hdr.njobs = (unsigned)pb.jobs.size();
    hdr.total = (unsigned)pb.blocks;
    std::memcpy(R.h_table[slot], &hdr, sizeof(hdr));
    std::memcpy(R.h_table[slot] + sizeof(hdr), pb.jobs.data(), pb.jobs.size() * sizeof(ccl::Job));
    if (!R.exec[slot] && (st = capture_slot(R, slot)) != CCL_OK) return st;
    if (cudaGraphLaunch(R.exec[slot], stream) != cudaSuccess) return CCL_ERR_CUDA;
    if (cudaEventRecord(R.done[slot], stream) != cudaSuccess) return CCL_ERR_CUDA;
    return CCL_OK;
}

void destroy_runner(Runner *R) {
    drop_graphs(*R);
    for (int i = 0; i < kRing; ++i) {
        if (R->done[i]) cudaEventDestroy(R->done[i]);
        if (R->h_table[i]) cudaFreeHost(R->h_table[i]);
    }
    if (R->d_table) cudaFree(R->d_table);
    if (R->d_ws) cudaFree(R->d_ws);
    if (R->capture) cudaStreamDestroy(R->capture);
    delete R;
}

// --- autotune cache ----------------------------------------------------------

std::mutex g_tmu;
std::map<std::string, int> g_tuned;
bool g_tuned_loaded = false;

std::string cache_path() {
    const char *p = std::getenv("CCL_AUTOTUNE_CACHE");
    if (p && *p) return p;
    const char *home = std::getenv("HOME");
    return std::string(home && *home ? home : "/tmp") + "/.cache/ccl_gb300/autotune.txt";
}

void load_cache_locked() {
    if (g_tuned_loaded) return;
    g_tuned_loaded = true;
    std::ifstream f(cache_path());
    std::string key;
    int geo;
    while (f >> key >> geo)
        if (geo >= 0 && geo < ccl::kNumGeo) g_tuned[key] = geo;
}

void store_cache_locked(const std::string &key, int geo) {
    g_tuned[key] = geo;
    const std::string path = cache_path();
    // create the parent folders one level at a time (best effort)
    for (size_t pos = path.find('/', 1); pos != std::string::npos; pos = path.find('/', pos + 1))
        mkdir(path.substr(0, pos).c_str(), 0755);
    std::ofstream f(path, std::ios::app);
    if (f) f << key << ' ' << geo << '\n';
}

// GPU name with blanks replaced, looked up once per device.
std::string device_name() {
    static std::mutex mu;
    static std::map<int, std::string> names;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    auto it = names.find(dev);
    if (it != names.end()) return it->second;
    cudaDeviceProp prop{};
    cudaGetDeviceProperties(&prop, dev);
    std::string name(prop.name);
    for (char &c : name)
        if (c == ' ') c = '_';
    names[dev] = name;
    return name;
}

std::string size_key(const ccl_image *images, int n, int conn) {
    const std::string name = device_name();
    double area = 0;
    int m = 0;
    for (int i = 0; i < n; ++i)
        if (images[i].H > 0 && images[i].W > 0) {
            area += (double)images[i].H * images[i].W;
            ++m;
        }
    const int cls = m ? (int)std::lround(std::log2(area / m)) : 0;
    return name + "|c" + std::to_string(conn) + "|s" + std::to_string(cls);
}

int env_tile() {
    const char *e = std::getenv("CCL_TILE");
    if (!e || !*e) return -1;
    for (int g = 0; g < ccl::kNumGeo; ++g)
        if (std::strcmp(e, ccl::geo_name(g)) == 0) return g;
    return -1;
}

ccl_status autotune(const ccl_image *images, int n, int conn, cudaStream_t stream, int *best_out) {
    float best_ms = 0.f;
    int best = -1;
    cudaEvent_t a = nullptr, b = nullptr;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return CCL_ERR_CUDA;
    ccl_status st = CCL_OK;
    for (int g = 0; g < ccl::kNumGeo && st == CCL_OK; ++g) {
        Prepared pb;
        if ((st = prepare(images, n, conn, g, pb)) != CCL_OK) break;
        if ((st = run_batch(pb, conn, g, stream)) != CCL_OK) break;  // warm-up, builds the graph
        std::vector<float> t;
        for (int rep = 0; rep < 3 && st == CCL_OK; ++rep) {
            cudaEventRecord(a, stream);
            st = run_batch(pb, conn, g, stream);
            cudaEventRecord(b, stream);
            if (cudaEventSynchronize(b) != cudaSuccess) st = CCL_ERR_CUDA;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, a, b);
            t.push_back(ms);
        }
        if (st != CCL_OK) break;
        std::sort(t.begin(), t.end());
        if (best < 0 || t[1] < best_ms) {
            best = g;
            best_ms = t[1];
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (st != CCL_OK) return st;
    if (best < 0) best = 0;
    {
        std::lock_guard<std::mutex> lk(g_tmu);
        store_cache_locked(size_key(images, n, conn), best);
    }
    // the batch is labelled with the chosen shape last
    Prepared pb;
    if ((st = prepare(images, n, conn, best, pb)) != CCL_OK) return st;
    if ((st = run_batch(pb, conn, best, stream)) != CCL_OK) return st;
    if (best_out) *best_out = best;
    return CCL_OK;
}

// Shape for this batch: $CCL_TILE, else the tuned one, else -1 (untuned).
int chosen_tile(const ccl_image *images, int n, int conn) {
    const int e = env_tile();
    if (e >= 0) return e;
    std::lock_guard<std::mutex> lk(g_tmu);
    load_cache_locked();
    const auto it = g_tuned.find(size_key(images, n, conn));
    return it == g_tuned.end() ? -1 : it->second;
}

}  // namespace

namespace ccl {

int release_batched_stream(int dev, cudaStream_t stream) {
    std::lock_guard<std::mutex> lk(g_bmu);
    int n = 0;
    for (auto it = g_runners.begin(); it != g_runners.end();) {
        if (std::get<0>(it->first) == dev && std::get<1>(it->first) == stream) {
            destroy_runner(it->second);
            it = g_runners.erase(it);
            ++n;
        } else {
            ++it;
        }
    }
    return n;
}

}  // namespace ccl

extern "C" {

int ccl_tile_count(void) { return ccl::kNumGeo; }

const char *ccl_tile_name(int tile) { return ccl::geo_name(tile); }

ccl_status ccl_label_batched_tile(const ccl_image *images, int n, int connectivity, int tile, void *stream) {
    if (tile < 0 || tile >= ccl::kNumGeo) return CCL_ERR_INVALID_ARG;
    Prepared pb;
    const ccl_status st = prepare(images, n, connectivity, tile, pb);
    if (st != CCL_OK) return st;
    return run_batch(pb, connectivity, tile, static_cast<cudaStream_t>(stream));
}

ccl_status ccl_autotune_batched(const ccl_image *images, int n, int connectivity, void *stream, int *tile) {
    Prepared pb;
    const ccl_status st = prepare(images, n, connectivity, 0, pb);
    if (st != CCL_OK) return st;
    if (pb.jobs.empty()) {
        if (tile) *tile = 0;
        return CCL_OK;
    }
    return autotune(images, n, connectivity, static_cast<cudaStream_t>(stream), tile);
}

ccl_status ccl_batched_tile(const ccl_image *images, int n, int connectivity, int *tile) {
    if (!tile || n < 0 || (n > 0 && !images) || (connectivity != 4 && connectivity != 8))
        return CCL_ERR_INVALID_ARG;
    *tile = chosen_tile(images, n, connectivity);
    return CCL_OK;
}

ccl_status ccl_label_batched(const ccl_image *images, int n, int connectivity, void *stream) {
    Prepared pb;
    ccl_status st = prepare(images, n, connectivity, 0, pb);
    if (st != CCL_OK || pb.jobs.empty()) return st;
    const int tile = chosen_tile(images, n, connectivity);
    if (tile < 0) return autotune(images, n, connectivity, static_cast<cudaStream_t>(stream), nullptr);
    if (tile != 0 && (st = prepare(images, n, connectivity, tile, pb)) != CCL_OK) return st;
    return run_batch(pb, connectivity, tile, static_cast<cudaStream_t>(stream));
}

}  // extern "C"
