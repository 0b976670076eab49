// ccl_server.cu -- continuous-batching labelling server behind the C ABI.
//
// Requests carry host frames.  A scheduler thread keeps them in arrival
// order and forms a batch from the front of the queue whenever a CUDA stream
// is idle: requests join while the batch is below max_batch, fewer than
// max_slots requests are on the device, their device buffers fit in the
// resident arena (the server's share of HBM, hbm_budget_bytes) and they have
// the connectivity of the batch's first request.  A batch is enqueued on its
// stream as: one host->device copy per frame, one batched labelling (graph
// replay of the persistent kernels), one device->host copy per frame and a
// host callback.  The callback hands the batch back to the scheduler, which
// frees its arena ranges (admitting waiting requests) and wakes the waiters.
// With several streams, copies of one batch overlap kernels of another.
//
// Latency of a request = time from ccl_server_submit() to the callback of
// its batch (labels are in host memory by then).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdint>
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

double seconds_since(Clock::time_point t0, Clock::time_point t) {
    return std::chrono::duration<double>(t - t0).count();
}

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
        bytes = (bytes + 255) & ~(size_t)255;
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
        bytes = (bytes + 255) & ~(size_t)255;
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

struct Request {
    uint64_t ticket = 0;
    const uint8_t *host_img = nullptr;
    int32_t *host_labels = nullptr;
    int H = 0, W = 0, conn = 8;
    size_t pitch = 0, dpitch = 0;
    size_t img_off = 0, lab_off = 0;
    Clock::time_point t_submit, t_done;
    bool done = false;
    ccl_status status = CCL_OK;
};

struct Batch {
    ccl_server *srv = nullptr;
    std::vector<Request *> reqs;
    int stream = 0;
};

}  // namespace

struct ccl_server {
    ccl_server_config cfg{};
    int device = 0;
    unsigned char *arena_base = nullptr;
    Arena arena;
    std::vector<cudaStream_t> streams;
    std::vector<bool> stream_busy;

    std::mutex mu;
    std::condition_variable cv_sched, cv_done;
    std::deque<Request *> pending;
    std::map<uint64_t, Request *> requests;
    std::deque<Batch *> finished;
    uint64_t next_ticket = 1;
    uint64_t events = 0;  // bumped by every submission and finished batch
    int on_device = 0;
    bool stop = false;
    std::thread sched;
    // block shape per connectivity (index 0: 4, 1: 8), fixed at the first
    // batch so that each stream keeps one graph runner whose capacity the
    // first full batches settle; -1 until then (scheduler thread only)
    int tile[2] = {-1, -1};

    // statistics
    Clock::time_point t_create, t_first_submit, t_last_done;
    bool any_submit = false;
    uint64_t submitted = 0, completed = 0, rejected = 0, pixels = 0;
    std::vector<double> latencies_ms;
};

namespace {

void CUDART_CB on_batch_done(void *p) {
    Batch *b = static_cast<Batch *>(p);
    ccl_server *s = b->srv;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->finished.push_back(b);
        ++s->events;
    }
    s->cv_sched.notify_one();
}

size_t image_bytes(const Request &r) { return r.dpitch * (size_t)r.H; }
size_t label_bytes(const Request &r) { return (size_t)r.H * (size_t)r.W * sizeof(int32_t); }

// Runs with s->mu held.  Hands finished batches back: frees their arena
// ranges and marks their requests done.
void reap_locked(ccl_server *s) {
    const Clock::time_point now = Clock::now();
    while (!s->finished.empty()) {
        Batch *b = s->finished.front();
        s->finished.pop_front();
        s->stream_busy[b->stream] = false;
        for (Request *r : b->reqs) {
            s->arena.release(r->img_off, image_bytes(*r));
            s->arena.release(r->lab_off, label_bytes(*r));
            r->done = true;
            r->t_done = now;
            --s->on_device;
            ++s->completed;
            s->pixels += (uint64_t)r->H * (uint64_t)r->W;
            s->latencies_ms.push_back(1e3 * std::chrono::duration<double>(now - r->t_submit).count());
            s->t_last_done = now;
        }
        delete b;
    }
    s->cv_done.notify_all();
}

// Runs with s->mu held: takes requests from the front of the queue for one
// batch on `stream`; returns null when nothing can be admitted now.
Batch *admit_locked(ccl_server *s, int stream) {
    Batch *b = nullptr;
    while (!s->pending.empty()) {
        Request *r = s->pending.front();
        if (b && ((int)b->reqs.size() >= s->cfg.max_batch || r->conn != b->reqs.front()->conn)) break;
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
        }
        b->reqs.push_back(r);
    }
    return b;
}

// Enqueues a batch (without the lock): copies in, labels, copies out, callback.
ccl_status launch(ccl_server *s, Batch *b) {
    cudaStream_t st = s->streams[b->stream];
    std::vector<ccl_image> imgs;
    imgs.reserve(b->reqs.size());
    for (Request *r : b->reqs) {
        uint8_t *dimg = s->arena_base + r->img_off;
        int32_t *dlab = reinterpret_cast<int32_t *>(s->arena_base + r->lab_off);
        if (cudaMemcpy2DAsync(dimg, r->dpitch, r->host_img, r->pitch, (size_t)r->W, (size_t)r->H,
                              cudaMemcpyHostToDevice, st) != cudaSuccess)
            return CCL_ERR_CUDA;
        imgs.push_back(ccl_image{dimg, dlab, r->H, r->W, r->dpitch});
    }
    int &tile = s->tile[b->reqs.front()->conn == 8 ? 1 : 0];
    if (tile < 0 &&
        (ccl_batched_tile(imgs.data(), (int)imgs.size(), b->reqs.front()->conn, &tile) != CCL_OK || tile < 0))
        tile = 0;
    ccl_status status =
        ccl_label_batched_tile(imgs.data(), (int)imgs.size(), b->reqs.front()->conn, tile, st);
    if (status != CCL_OK) return status;
    for (Request *r : b->reqs) {
        if (cudaMemcpyAsync(r->host_labels, s->arena_base + r->lab_off, label_bytes(*r), cudaMemcpyDeviceToHost,
                            st) != cudaSuccess)
            return CCL_ERR_CUDA;
    }
    if (cudaLaunchHostFunc(st, on_batch_done, b) != cudaSuccess) return CCL_ERR_CUDA;
    return CCL_OK;
}

void scheduler(ccl_server *s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (true) {
        reap_locked(s);
        if (s->stop && s->pending.empty() && s->on_device == 0) break;
        bool launched = false;
        for (int i = 0; i < (int)s->streams.size() && !s->stop; ++i) {
            if (s->stream_busy[i]) continue;
            Batch *b = admit_locked(s, i);
            if (!b) break;
            s->stream_busy[i] = true;
            lk.unlock();
            const ccl_status st = launch(s, b);
            lk.lock();
            if (st != CCL_OK) {
                // the batch never reaches its callback: let whatever was
                // enqueued drain, then fail its requests here
                lk.unlock();
                cudaStreamSynchronize(s->streams[i]);
                lk.lock();
                s->stream_busy[i] = false;
                for (Request *r : b->reqs) {
                    s->arena.release(r->img_off, image_bytes(*r));
                    s->arena.release(r->lab_off, label_bytes(*r));
                    r->status = st;
                    r->done = true;
                    --s->on_device;
                }
                delete b;
                s->cv_done.notify_all();
            }
            launched = true;
        }
        if (s->stop && s->on_device == 0) {
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
            // (a submission or a finished batch); the wait releases the lock,
            // which the completion callback needs
            const uint64_t seen = s->events;
            s->cv_sched.wait_for(lk, std::chrono::milliseconds(5), [&] { return s->events != seen; });
        }
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
    s->stream_busy.assign(config->n_streams, false);
    for (auto &st : s->streams) {
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            cudaFree(s->arena_base);
            delete s;
            return CCL_ERR_CUDA;
        }
    }
    s->t_create = Clock::now();
    s->sched = std::thread(scheduler, s);
    *out = s;
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
        // a frame that could never fit the arena is refused outright
        if (((image_bytes(*r) + 255) & ~(size_t)255) + ((label_bytes(*r) + 255) & ~(size_t)255) > s->arena.size()) {
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
        std::vector<double> v = s->latencies_ms;
        std::sort(v.begin(), v.end());
        const auto pct = [&](double q) {
            const size_t i = std::min(v.size() - 1, (size_t)(q * (double)(v.size() - 1) + 0.5));
            return v[i];
        };
        double sum = 0;
        for (double x : v) sum += x;
        st.p50_ms = pct(0.50);
        st.p99_ms = pct(0.99);
        st.max_ms = v.back();
        st.mean_ms = sum / (double)v.size();
        const double span = seconds_since(s->t_first_submit, s->t_last_done);
        st.gpixel_s = span > 0 ? (double)s->pixels / span / 1e9 : 0.0;
    }
    *out = st;
    return CCL_OK;
}

ccl_status ccl_server_reset_stats(ccl_server *s) {
    if (!s) return CCL_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    s->latencies_ms.clear();
    s->submitted = s->completed = s->rejected = s->pixels = 0;
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
    for (auto &st : s->streams) {
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
    for (auto &kv : s->requests) delete kv.second;
    cudaFree(s->arena_base);
    delete s;
}

}  // extern "C"
