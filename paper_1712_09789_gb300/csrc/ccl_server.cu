// ccl_server.cu -- continuous-batching labelling server behind the C ABI.
//
// Requests carry host frames.  A scheduler thread keeps them in arrival
// order and forms a batch from the front of the queue whenever a CUDA stream
// is idle: requests join while the batch is below max_batch, fewer than
// max_slots requests are on the device, their device buffers and the batch's
// scratch fit in the resident arena (the server's share of HBM,
// hbm_budget_bytes) and they have the connectivity of the batch's first
// request.  Every byte the server uses on the device comes from that arena:
// frames, labels, the batch's job table and its labelling scratch.
//
// A batch is enqueued on its stream as: one host->device copy per frame, the
// job table copy, the three labelling kernels over all blocks of the batch
// (persistent grids pulling blocks from a device work counter), then one
// device->host copy per frame in increasing size, each followed by an event.
// A completion thread per stream waits on those events in order (blocking
// synchronisation, so it sleeps) and completes each request as soon as its
// own labels are in host memory: a small frame does not wait for a large
// frame's copy-out, and the GPU never waits for the host.  When the batch's
// last event has passed, the thread retires the batch: it frees its arena
// ranges and hands the stream back to the scheduler.  No CUDA call is made
// while the server's lock is held.  With several streams, copies of one batch
// overlap kernels of another.
//
// Latency of a request = time from ccl_server_submit() until its completion
// thread has seen its label copy finish (labels are in host memory by then).
// Per batch, CUDA events split the device side into copy-in, labelling and
// copy-out.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/ccl.h"
#include "ccl_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b) {
    return 1e3 * std::chrono::duration<double>(b - a).count();
}

size_t up256(size_t v) { return (v + 255) & ~(size_t)255; }

// First-fit allocator over one device arena; ranges are 256-byte aligned.
class Arena {
  public:
    void reset(size_t bytes) {
        free_.clear();
        free_[0] = bytes;
        size_ = bytes;
        used_ = 0;
    }
    bool alloc(size_t bytes, size_t &off) {
        bytes = up256(bytes);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                off = it->first;
                const size_t rest = it->second - bytes;
                const size_t start = it->first + bytes;
                free_.erase(it);
                if (rest) free_[start] = rest;
                used_ += bytes;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes) {
        bytes = up256(bytes);
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t size() const { return size_; }
    size_t used() const { return used_; }

  private:
    std::map<size_t, size_t> free_;
    size_t size_ = 0, used_ = 0;
};

struct Batch;

struct Request {
    uint64_t ticket = 0;
    const uint8_t *host_img = nullptr;
    int32_t *host_labels = nullptr;
    int H = 0, W = 0, conn = 8;
    size_t pitch = 0, dpitch = 0;
    size_t img_off = 0, lab_off = 0;
    Batch *batch = nullptr;
    Clock::time_point t_submit, t_admit, t_done;
    bool done = false;     // visible to waiters
    ccl_status status = CCL_OK;
};

struct Batch {
    ccl_server *srv = nullptr;
    std::vector<Request *> reqs;
    int stream = 0;
    int geo = 0;
    size_t blocks = 0;
    size_t ws_off = 0, ws_bytes = 0;   // labelling scratch
    size_t tab_off = 0, tab_bytes = 0; // job table
    std::vector<int> order;            // copy-out order (indices into reqs)
};

// Per-stream state: the stream, page-locked staging of the job table, the
// events that split a batch into copy-in, labelling and copy-out, one event
// per request's label copy, and the completion thread that watches them.
struct StreamCtx {
    cudaStream_t s = nullptr;
    bool busy = false;
    unsigned char *h_table = nullptr;
    size_t h_table_bytes = 0;
    cudaEvent_t ev[4] = {};
    std::vector<cudaEvent_t> req_ev;
    Batch *watch = nullptr;            // the batch its thread waits on
    std::condition_variable cv;
    std::thread waiter;
};

// Percentile q of v (sorted copy).
double pct(std::vector<double> v, double q) {
    if (v.empty()) return 0.0;
    std::sort(v.begin(), v.end());
    const size_t i = std::min(v.size() - 1, (size_t)(q * (double)(v.size() - 1) + 0.5));
    return v[i];
}

}  // namespace

struct ccl_server {
    ccl_server_config cfg{};
    int device = 0;
    unsigned char *arena_base = nullptr;
    Arena arena;
    std::deque<StreamCtx> streams;     // (a deque: StreamCtx is not movable)
    bool quit_waiters = false;

    std::mutex mu;
    std::condition_variable cv_sched, cv_done;
    std::deque<Request *> pending;
    std::map<uint64_t, Request *> requests;
    uint64_t next_ticket = 1;
    uint64_t events = 0;  // bumped by every submission and completion
    int on_device = 0;
    int batches_on_device = 0;
    bool stop = false;
    std::thread sched;
    // block shape per connectivity (index 0: 4, 1: 8), fixed at the first
    // batch of that connectivity (scheduler thread only); -1 until then
    int tile[2] = {-1, -1};

    // statistics
    Clock::time_point t_first_submit, t_last_done;
    bool any_submit = false;
    uint64_t submitted = 0, completed = 0, rejected = 0, pixels = 0, batches = 0, multi_batches = 0;
    uint64_t overlapped = 0;
    int max_batch_seen = 0, max_batches_in_flight = 0;
    std::vector<double> latencies_ms, queue_ms, h2d_ms, label_ms, d2h_ms;
    // device spans [copy-in start, copy-out end] of recently retired batches,
    // in ms after `t0_event` (recorded once at creation)
    cudaEvent_t t0_event = nullptr;
    std::deque<std::pair<float, float>> recent_spans;
};

namespace {

size_t image_bytes(const Request &r) { return r.dpitch * (size_t)r.H; }
size_t label_bytes(const Request &r) { return (size_t)r.H * (size_t)r.W * sizeof(int32_t); }
size_t table_bytes(size_t jobs) { return sizeof(ccl::JobHeader) + jobs * sizeof(ccl::Job); }

// Largest labelling scratch any block shape needs for an H x W frame.
size_t frame_scratch_bytes(int H, int W) {
    size_t m = 0;
    for (int g = 0; g < ccl::kNumGeo; ++g)
        m = std::max(m, ccl::geo_workspace_bytes(g, ccl::geo_blocks(g, H, W)));
    return m;
}

// Arena bytes that one frame served alone needs: image, labels, scratch and
// a one-entry job table, each rounded to the arena's 256-byte granule.
size_t lone_frame_bytes(int H, int W) {
    const size_t dpitch = ((size_t)W + 15) & ~(size_t)15;
    return up256(dpitch * (size_t)H) + up256((size_t)H * (size_t)W * sizeof(int32_t)) +
           up256(frame_scratch_bytes(H, W)) + up256(table_bytes(1));
}

// Runs with s->mu held: request r's labels are in host memory.
void complete_locked(ccl_server *s, Request *r, Clock::time_point now) {
    s->arena.release(r->img_off, image_bytes(*r));
    s->arena.release(r->lab_off, label_bytes(*r));
    r->t_done = now;
    r->done = true;
    --s->on_device;
    ++s->completed;
    s->pixels += (uint64_t)r->H * (uint64_t)r->W;
    s->latencies_ms.push_back(ms_between(r->t_submit, now));
    s->t_last_done = now;
}

// Completion thread of stream `i`: waits (sleeping) on the events of the
// batch it is given, completes each request when its label copy is done, and
// retires the batch after its last event.
void waiter(ccl_server *s, int i) {
    cudaSetDevice(s->device);
    StreamCtx &c = s->streams[i];
    std::unique_lock<std::mutex> lk(s->mu);
    while (true) {
        c.cv.wait(lk, [&] { return c.watch != nullptr || s->quit_waiters; });
        if (!c.watch) break;
        Batch *b = c.watch;
        lk.unlock();
        for (size_t k = 0; k < b->order.size(); ++k) {
            const bool ok = cudaEventSynchronize(c.req_ev[k]) == cudaSuccess;
            const Clock::time_point now = Clock::now();
            {
                std::lock_guard<std::mutex> g(s->mu);
                Request *r = b->reqs[b->order[k]];
                if (!ok) r->status = CCL_ERR_CUDA;
                complete_locked(s, r, now);
                ++s->events;
            }
            s->cv_done.notify_all();
            s->cv_sched.notify_one();
        }
        // stage times and the device span of the batch (no lock held)
        float t01 = 0.f, t12 = 0.f, t23 = 0.f, a = 0.f, e = 0.f;
        bool ok = cudaEventSynchronize(c.ev[3]) == cudaSuccess;
        ok = ok && cudaEventElapsedTime(&t01, c.ev[0], c.ev[1]) == cudaSuccess &&
             cudaEventElapsedTime(&t12, c.ev[1], c.ev[2]) == cudaSuccess &&
             cudaEventElapsedTime(&t23, c.ev[2], c.ev[3]) == cudaSuccess &&
             cudaEventElapsedTime(&a, s->t0_event, c.ev[0]) == cudaSuccess &&
             cudaEventElapsedTime(&e, s->t0_event, c.ev[3]) == cudaSuccess;
        if (!ok) cudaGetLastError();
        lk.lock();
        if (ok) {
            for (size_t k = 0; k < b->reqs.size(); ++k) {
                s->h2d_ms.push_back(t01);
                s->label_ms.push_back(t12);
                s->d2h_ms.push_back(t23);
            }
            bool overlap = false;
            for (const auto &sp : s->recent_spans)
                if (sp.first < e && a < sp.second) overlap = true;
            if (overlap) ++s->overlapped;
            s->recent_spans.emplace_back(a, e);
            if (s->recent_spans.size() > 64) s->recent_spans.pop_front();
        }
        s->arena.release(b->ws_off, b->ws_bytes);
        s->arena.release(b->tab_off, b->tab_bytes);
        c.busy = false;
        c.watch = nullptr;
        --s->batches_on_device;
        ++s->events;
        delete b;
        s->cv_sched.notify_one();
    }
}

// Gives the last request of batch b back to the front of the queue.
void unadmit_last_locked(ccl_server *s, Batch *b) {
    Request *r = b->reqs.back();
    b->reqs.pop_back();
    b->blocks -= ccl::geo_blocks(b->geo, r->H, r->W);
    s->arena.release(r->img_off, image_bytes(*r));
    s->arena.release(r->lab_off, label_bytes(*r));
    r->batch = nullptr;
    --s->on_device;
    s->pending.push_front(r);
}

// Block shape for a connectivity, fixed at its first batch: the tuned one for
// that frame size if the autotuner has one, else the 512x64 blocks.
int tile_for(ccl_server *s, const Request &r) {
    int &tile = s->tile[r.conn == 8 ? 1 : 0];
    if (tile < 0) {
        const ccl_image im{r.host_img, r.host_labels, r.H, r.W, r.pitch};
        // untuned: the piece labeller's 512x64 blocks
        if (ccl_batched_tile(&im, 1, r.conn, &tile) != CCL_OK || tile < 0 || tile >= ccl::kNumGeo) tile = 4;
    }
    return tile;
}

// Runs with s->mu held: takes requests from the front of the queue for one
// batch on `stream`, with frames, scratch and job table carved from the
// arena; returns null when nothing can be admitted now.
Batch *admit_locked(ccl_server *s, int stream) {
    if (s->pending.empty()) return nullptr;
    const int conn = s->pending.front()->conn;
    const int geo = tile_for(s, *s->pending.front());
    Batch *b = nullptr;
    const Clock::time_point now = Clock::now();
    while (!s->pending.empty()) {
        Request *r = s->pending.front();
        if (b && ((int)b->reqs.size() >= s->cfg.max_batch || r->conn != conn)) break;
        if (s->on_device >= s->cfg.max_slots) break;
        size_t io = 0, lo = 0;
        if (!s->arena.alloc(image_bytes(*r), io)) break;
        if (!s->arena.alloc(label_bytes(*r), lo)) {
            s->arena.release(io, image_bytes(*r));
            break;
        }
        r->img_off = io;
        r->lab_off = lo;
        s->pending.pop_front();
        ++s->on_device;
        if (!b) {
            b = new Batch();
            b->srv = s;
            b->stream = stream;
            b->geo = geo;
        }
        r->batch = b;
        r->t_admit = now;
        b->reqs.push_back(r);
        b->blocks += ccl::geo_blocks(geo, r->H, r->W);
    }
    if (!b) return nullptr;
    // the batch's scratch and job table; drop requests from its end until
    // they fit (a frame alone always fits an empty arena: submit checks it)
    while (true) {
        b->ws_bytes = ccl::geo_workspace_bytes(geo, b->blocks);
        b->tab_bytes = table_bytes(b->reqs.size());
        if (s->arena.alloc(b->ws_bytes, b->ws_off)) {
            if (s->arena.alloc(b->tab_bytes, b->tab_off)) break;
            s->arena.release(b->ws_off, b->ws_bytes);
        }
        unadmit_last_locked(s, b);
        if (b->reqs.empty()) {
            delete b;
            return nullptr;
        }
    }
    for (Request *r : b->reqs) s->queue_ms.push_back(ms_between(r->t_submit, r->t_admit));
    return b;
}

// Enqueues a batch (without the lock): copies in, job table, the three
// labelling kernels, copies out (smallest first) with a callback after each,
// and the batch's final callback.
ccl_status launch(ccl_server *s, Batch *b) {
    StreamCtx &c = s->streams[b->stream];
    cudaStream_t st = c.s;
    unsigned char *base = s->arena_base;
    if (cudaEventRecord(c.ev[0], st) != cudaSuccess) return CCL_ERR_CUDA;
    ccl::JobHeader hdr{};
    hdr.njobs = (unsigned)b->reqs.size();
    hdr.total = (unsigned)b->blocks;
    std::memcpy(c.h_table, &hdr, sizeof(hdr));
    ccl::Job *jobs = reinterpret_cast<ccl::Job *>(c.h_table + sizeof(hdr));
    int bw = 0, bh = 0;
    ccl::geo_block_shape(b->geo, &bw, &bh);
    unsigned block0 = 0;
    for (size_t k = 0; k < b->reqs.size(); ++k) {
        Request *r = b->reqs[k];
        uint8_t *dimg = base + r->img_off;
        int32_t *dlab = reinterpret_cast<int32_t *>(base + r->lab_off);
        if (cudaMemcpy2DAsync(dimg, r->dpitch, r->host_img, r->pitch, (size_t)r->W, (size_t)r->H,
                              cudaMemcpyHostToDevice, st) != cudaSuccess)
            return CCL_ERR_CUDA;
        ccl::Job &j = jobs[k];
        j.img = dimg;
        j.labels = dlab;
        j.pitch = r->dpitch;
        j.H = r->H;
        j.W = r->W;
        j.nbx = (r->W + bw - 1) / bw;
        j.nby = (r->H + bh - 1) / bh;
        j.block0 = block0;
        j.key0 = 0;
        j.pad = 0;
        // arena ranges are 256-byte aligned and dpitch a multiple of 16
        j.flags = ccl::kJobVecIn | ((r->W & 3) == 0 ? ccl::kJobVecOut : 0u);
        block0 += (unsigned)j.nbx * (unsigned)j.nby;
    }
    if (cudaEventRecord(c.ev[1], st) != cudaSuccess) return CCL_ERR_CUDA;
    unsigned char *dtab = base + b->tab_off;
    if (cudaMemcpyAsync(dtab, c.h_table, b->tab_bytes, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return CCL_ERR_CUDA;
    if (ccl::launch_jobs(b->geo, b->reqs.front()->conn, reinterpret_cast<ccl::JobHeader *>(dtab),
                         reinterpret_cast<const ccl::Job *>(dtab + sizeof(ccl::JobHeader)), base + b->ws_off,
                         b->blocks, st, ccl::iteration_cap_api()) != 0)
        return CCL_ERR_CUDA;
    if (cudaEventRecord(c.ev[2], st) != cudaSuccess) return CCL_ERR_CUDA;
    std::vector<int> &order = b->order;
    order.resize(b->reqs.size());
    for (size_t k = 0; k < order.size(); ++k) order[k] = (int)k;
    std::stable_sort(order.begin(), order.end(),
                     [&](int x, int y) { return label_bytes(*b->reqs[x]) < label_bytes(*b->reqs[y]); });
    for (size_t k = 0; k < order.size(); ++k) {
        Request *r = b->reqs[order[k]];
        if (cudaMemcpyAsync(r->host_labels, base + r->lab_off, label_bytes(*r), cudaMemcpyDeviceToHost, st) !=
                cudaSuccess ||
            cudaEventRecord(c.req_ev[k], st) != cudaSuccess)
            return CCL_ERR_CUDA;
    }
    if (cudaEventRecord(c.ev[3], st) != cudaSuccess) return CCL_ERR_CUDA;
    return CCL_OK;
}

// Runs with s->mu held (released around the stream wait): a batch whose
// enqueue failed is never given to its completion thread.  Waits for what
// was enqueued, then fails every request of the batch.
void fail_batch_locked(ccl_server *s, Batch *b, ccl_status st, std::unique_lock<std::mutex> &lk) {
    lk.unlock();
    cudaStreamSynchronize(s->streams[b->stream].s);
    cudaGetLastError();
    lk.lock();
    for (Request *r : b->reqs) {
        s->arena.release(r->img_off, image_bytes(*r));
        s->arena.release(r->lab_off, label_bytes(*r));
        r->status = st;
        r->done = true;
        --s->on_device;
    }
    s->arena.release(b->ws_off, b->ws_bytes);
    s->arena.release(b->tab_off, b->tab_bytes);
    s->streams[b->stream].busy = false;
    --s->batches_on_device;
    delete b;
    s->cv_done.notify_all();
}

void scheduler(ccl_server *s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (true) {
        if (s->stop && s->pending.empty() && s->batches_on_device == 0) break;
        bool launched = false;
        for (int i = 0; i < (int)s->streams.size() && !s->stop; ++i) {
            if (s->streams[i].busy) continue;
            Batch *b = admit_locked(s, i);
            if (!b) break;
            s->streams[i].busy = true;
            ++s->batches_on_device;
            ++s->batches;
            if (b->reqs.size() > 1) ++s->multi_batches;
            s->max_batch_seen = std::max(s->max_batch_seen, (int)b->reqs.size());
            s->max_batches_in_flight = std::max(s->max_batches_in_flight, s->batches_on_device);
            lk.unlock();
            const ccl_status st = launch(s, b);
            lk.lock();
            if (st != CCL_OK) {
                fail_batch_locked(s, b, st, lk);
            } else {
                s->streams[i].watch = b;
                s->streams[i].cv.notify_one();
            }
            launched = true;
        }
        if (s->stop && s->batches_on_device == 0) {
            // drop what was never admitted
            for (Request *r : s->pending) {
                r->status = CCL_ERR_BUSY;
                r->done = true;
            }
            s->pending.clear();
            s->cv_done.notify_all();
            continue;
        }
        if (!launched) {
            // everything admissible was started: sleep until something changes
            // (a submission or a completion); the wait releases the lock, which
            // the completion threads need
            const uint64_t seen = s->events;
            s->cv_sched.wait_for(lk, std::chrono::milliseconds(5), [&] { return s->events != seen; });
        }
    }
}

// Stops the completion threads (after the scheduler has ended, so no batch
// is on the device) and frees the per-stream resources.
void destroy_streams(ccl_server *s) {
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->quit_waiters = true;
    }
    for (auto &c : s->streams) c.cv.notify_all();
    for (auto &c : s->streams)
        if (c.waiter.joinable()) c.waiter.join();
    for (auto &c : s->streams) {
        if (c.s) {
            cudaStreamSynchronize(c.s);
            cudaStreamDestroy(c.s);
        }
        for (auto &e : c.ev)
            if (e) cudaEventDestroy(e);
        for (auto &e : c.req_ev)
            if (e) cudaEventDestroy(e);
        if (c.h_table) cudaFreeHost(c.h_table);
        c.s = nullptr;
        c.h_table = nullptr;
        c.req_ev.clear();
        for (auto &e : c.ev) e = nullptr;
    }
}

}  // namespace

extern "C" {

ccl_status ccl_server_create(const ccl_server_config *config, ccl_server **out) {
    if (!config || !out) return CCL_ERR_INVALID_ARG;
    if (config->max_slots < 1 || config->n_streams < 1 || config->n_streams > 16 || config->max_batch < 1 ||
        config->hbm_budget_bytes < (1u << 20))
        return CCL_ERR_INVALID_ARG;
    ccl_server *s = new ccl_server();
    s->cfg = *config;
    s->device = config->device;
    if (cudaSetDevice(s->device) != cudaSuccess) {
        delete s;
        return CCL_ERR_CUDA;
    }
    if (cudaMalloc(&s->arena_base, config->hbm_budget_bytes) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return CCL_ERR_OUT_OF_MEMORY;
    }
    s->arena.reset(config->hbm_budget_bytes);
    s->streams.resize(config->n_streams);
    bool ok = cudaEventCreate(&s->t0_event) == cudaSuccess;
    for (auto &c : s->streams) {
        ok = ok && cudaStreamCreateWithFlags(&c.s, cudaStreamNonBlocking) == cudaSuccess;
        // the completion thread sleeps in its waits (blocking synchronisation)
        for (auto &e : c.ev) ok = ok && cudaEventCreateWithFlags(&e, cudaEventBlockingSync) == cudaSuccess;
        c.req_ev.assign((size_t)config->max_batch, nullptr);
        for (auto &e : c.req_ev)
            ok = ok && cudaEventCreateWithFlags(&e, cudaEventBlockingSync | cudaEventDisableTiming) == cudaSuccess;
        c.h_table_bytes = table_bytes((size_t)config->max_batch);
        ok = ok && cudaMallocHost(&c.h_table, c.h_table_bytes) == cudaSuccess;
    }
    ok = ok && cudaEventRecord(s->t0_event, s->streams[0].s) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        destroy_streams(s);
        if (s->t0_event) cudaEventDestroy(s->t0_event);
        cudaFree(s->arena_base);
        delete s;
        return CCL_ERR_CUDA;
    }
    for (int i = 0; i < (int)s->streams.size(); ++i) s->streams[i].waiter = std::thread(waiter, s, i);
    s->sched = std::thread(scheduler, s);
    *out = s;
    return CCL_OK;
}

ccl_status ccl_server_frame_bytes(int H, int W, size_t *bytes) {
    if (!bytes || H < 1 || W < 1) return CCL_ERR_INVALID_ARG;
    if ((long long)H * (long long)W > 2147483646LL) return CCL_ERR_UNSUPPORTED;
    *bytes = lone_frame_bytes(H, W);
    return CCL_OK;
}

ccl_status ccl_server_submit(ccl_server *s, const uint8_t *host_img, int H, int W, size_t pitch,
                             int connectivity, int32_t *host_labels, uint64_t *ticket) {
    if (!s || !ticket) return CCL_ERR_INVALID_ARG;
    ccl_status st = ccl::check_image_args_api(host_img, H, W, pitch, connectivity, host_labels);
    if (st != CCL_OK) return st;
    if (H == 0 || W == 0) return CCL_ERR_INVALID_ARG;
    Request *r = new Request();
    r->host_img = host_img;
    r->host_labels = host_labels;
    r->H = H;
    r->W = W;
    r->pitch = pitch;
    r->dpitch = ((size_t)W + 15) & ~(size_t)15;
    r->conn = connectivity;
    r->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        // a frame that could never fit the arena, even alone, is refused
        if (lone_frame_bytes(H, W) > s->arena.size()) {
            ++s->rejected;
            delete r;
            return CCL_ERR_UNSUPPORTED;
        }
        if (s->stop) {
            delete r;
            return CCL_ERR_BUSY;
        }
        r->ticket = s->next_ticket++;
        s->requests[r->ticket] = r;
        s->pending.push_back(r);
        ++s->events;
        if (!s->any_submit) {
            s->any_submit = true;
            s->t_first_submit = r->t_submit;
        }
        ++s->submitted;
        *ticket = r->ticket;
    }
    s->cv_sched.notify_one();
    return CCL_OK;
}

ccl_status ccl_server_poll(ccl_server *s, uint64_t ticket) {
    if (!s) return CCL_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->requests.find(ticket);
    if (it == s->requests.end()) return CCL_ERR_NOT_FOUND;
    return it->second->done ? it->second->status : CCL_ERR_BUSY;
}

ccl_status ccl_server_wait(ccl_server *s, uint64_t ticket, int timeout_ms) {
    if (!s) return CCL_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->requests.find(ticket);
    if (it == s->requests.end()) return CCL_ERR_NOT_FOUND;
    Request *r = it->second;
    const auto pred = [&] { return r->done; };
    if (timeout_ms < 0) {
        s->cv_done.wait(lk, pred);
    } else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), pred)) {
        return CCL_ERR_BUSY;
    }
    const ccl_status st = r->status;
    s->requests.erase(it);
    delete r;
    return st;
}

ccl_status ccl_server_stats(ccl_server *s, ccl_server_stats_t *out) {
    if (!s || !out) return CCL_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    ccl_server_stats_t st{};
    st.submitted = s->submitted;
    st.completed = s->completed;
    st.rejected = s->rejected;
    st.in_flight = s->on_device;
    st.queued = (int)s->pending.size();
    st.pixels = s->pixels;
    st.arena_bytes = s->arena.size();
    st.arena_used_bytes = s->arena.used();
    if (!s->latencies_ms.empty()) {
        double sum = 0;
        for (double x : s->latencies_ms) sum += x;
        st.p50_ms = pct(s->latencies_ms, 0.50);
        st.p99_ms = pct(s->latencies_ms, 0.99);
        st.max_ms = *std::max_element(s->latencies_ms.begin(), s->latencies_ms.end());
        st.mean_ms = sum / (double)s->latencies_ms.size();
        const double span = ms_between(s->t_first_submit, s->t_last_done) / 1e3;
        st.gpixel_s = span > 0 ? (double)s->pixels / span / 1e9 : 0.0;
    }
    st.queue_p50_ms = pct(s->queue_ms, 0.50);
    st.queue_p99_ms = pct(s->queue_ms, 0.99);
    st.h2d_p50_ms = pct(s->h2d_ms, 0.50);
    st.h2d_p99_ms = pct(s->h2d_ms, 0.99);
    st.label_p50_ms = pct(s->label_ms, 0.50);
    st.label_p99_ms = pct(s->label_ms, 0.99);
    st.d2h_p50_ms = pct(s->d2h_ms, 0.50);
    st.d2h_p99_ms = pct(s->d2h_ms, 0.99);
    st.batches = s->batches;
    st.multi_request_batches = s->multi_batches;
    st.overlapped_batches = s->overlapped;
    st.max_batch_requests = s->max_batch_seen;
    st.max_batches_in_flight = s->max_batches_in_flight;
    *out = st;
    return CCL_OK;
}

ccl_status ccl_server_reset_stats(ccl_server *s) {
    if (!s) return CCL_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    s->latencies_ms.clear();
    s->queue_ms.clear();
    s->h2d_ms.clear();
    s->label_ms.clear();
    s->d2h_ms.clear();
    s->submitted = s->completed = s->rejected = s->pixels = 0;
    s->batches = s->multi_batches = s->overlapped = 0;
    s->max_batch_seen = 0;
    s->max_batches_in_flight = s->batches_on_device;
    s->any_submit = false;
    return CCL_OK;
}

void ccl_server_destroy(ccl_server *s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        ++s->events;
    }
    s->cv_sched.notify_one();
    if (s->sched.joinable()) s->sched.join();
    destroy_streams(s);
    if (s->t0_event) cudaEventDestroy(s->t0_event);
    for (auto &kv : s->requests) delete kv.second;
    cudaFree(s->arena_base);
    delete s;
}

}  // extern "C"
