// Continuous-batching serving loop for batched X-drop extension.
//
// A request is a host batch (pools, seeds, scalars, result buffer).  The
// server owns one device arena of `budget_bytes` (one cudaMalloc at
// creation) and `max_inflight` slots, each a CUDA stream.  A scheduler
// thread admits queued requests in arrival order as soon as a slot is idle
// and the arena has room for the request's device copy (pools, seeds,
// results, workspace): it enqueues the host->device copies, the extension
// pipeline (logan_extend_batch) and the device->host copy of the results on
// the slot's stream, followed by a host callback that marks the request
// done and returns its arena bytes.  Requests on different slots run
// concurrently on the GPU: a new request is admitted while others are
// still executing, its kernels start as the running ones' persistent grids
// drain, and results do not depend on what else is in flight (each request
// has its own workspace).  The paper retrieves results asynchronously as
// kernels complete (Sec. IV-B); this is that idea for a stream of batches.
//
// Host side, a request's inputs and results pass through a pinned staging
// arena owned by the server: a copy between the device and pageable memory
// would block the scheduler thread until the slot's stream drained (a
// device->host copy into pageable memory returns only once it has run), so
// every request would wait for the previous one.  The scheduler copies the
// inputs into the staging area before enqueueing, the stream copies the
// results into it, and the completion callback copies them to the caller's
// buffer.  A request whose host buffers are all pinned already, or whose
// host bytes exceed the whole staging arena, is copied directly (for the
// latter, with pageable buffers, the scheduler waits for its copies).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/logan.h"

namespace {

constexpr size_t kAlign = 256;
inline size_t up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

// First-fit allocator over [0, size) with coalescing frees.
class Arena {
   public:
    void init(size_t size) {
        size_ = size;
        free_.clear();
        if (size) free_[0] = size;
        used_ = peak_ = 0;
    }
    bool alloc(size_t n, size_t* off) {
        n = up(std::max<size_t>(n, 1));
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= n) {
                *off = it->first;
                const size_t rest = it->second - n;
                const size_t at = it->first + n;
                free_.erase(it);
                if (rest) free_[at] = rest;
                used_ += n;
                peak_ = std::max(peak_, used_);
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t n) {
        n = up(std::max<size_t>(n, 1));
        used_ -= n;
        auto it = free_.emplace(off, n).first;
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
    size_t peak() const { return peak_; }

   private:
    size_t size_ = 0, used_ = 0, peak_ = 0;
    std::map<size_t, size_t> free_;
};

enum class St { Queued, Running, Done, Cancelled, Failed };

struct Req {
    logan_request_t r{};
    size_t bytes = 0;
    size_t ws_bytes = 0;
    size_t hbytes = 0;    // pinned staging bytes (0: copied directly)
    size_t hoff = 0;
    St state = St::Queued;
    int status = LOGAN_OK;
    size_t off = 0;
    int slot = -1;
    double t_submit = 0, t_admit = 0, t_done = 0;
};

struct Slot {
    cudaStream_t stream = nullptr;
    uint64_t ticket = 0;  // 0 = idle
};

size_t pool_bytes(const logan_seqs_t& p) {
    const size_t b = p.packed2bit ? ((p.pool_bases + 15) / 16 + 1) * 4 : p.pool_bases;
    return up(b) + up(size_t(p.count) * 8) + up(size_t(p.count) * 4);
}

// bytes of the caller's pool buffer (ASCII: pool_bases bytes; packed: the
// words up to ceil(pool_bases / 16))
size_t pool_host_bytes(const logan_seqs_t& p) {
    return p.packed2bit ? ((p.pool_bases + 15) / 16) * 4 : p.pool_bases;
}

size_t request_host_bytes(const logan_request_t& r) {
    size_t b = 0;
    for (const logan_seqs_t* p : {&r.A, &r.B}) {
        if (p == &r.B && r.same_pool) break;
        b += up(pool_host_bytes(*p)) + up(size_t(p->count) * 8) + up(size_t(p->count) * 4);
    }
    return b + up(size_t(r.n_pairs) * sizeof(logan_seed_t)) +
           (r.X_per_pair ? up(size_t(r.n_pairs) * 4) : 0) +
           up(size_t(r.n_pairs) * sizeof(logan_result_t));
}

bool is_pinned(const void* p) {
    if (!p) return true;
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeHost;
}

bool request_pinned(const logan_request_t& r) {
    for (const logan_seqs_t* p : {&r.A, &r.B})
        if (!is_pinned(p->bases) || !is_pinned(p->offsets) || !is_pinned(p->lengths)) return false;
    return is_pinned(r.seeds) && is_pinned(r.X_per_pair) && is_pinned(r.results);
}

// pinned staging capacity for a device budget: an eighth of it, within
// [16 MiB, 1 GiB] (host bytes are the inputs and results only; the device
// bytes also hold the workspace)
size_t staging_bytes(size_t budget) {
    return std::min<size_t>(std::max<size_t>(budget / 8, size_t(16) << 20), size_t(1) << 30);
}

}  // namespace

struct logan_server {
    logan_ctx_t* ctx = nullptr;
    int device = 0;
    char* dev = nullptr;
    Arena arena;
    char* host = nullptr;  // pinned staging
    Arena harena;
    std::vector<Slot> slots;
    std::mutex mu;
    std::condition_variable cv;       // scheduler wake-up
    std::condition_variable done_cv;  // waiters
    std::deque<uint64_t> queue;
    std::unordered_map<uint64_t, Req> reqs;
    uint64_t next_ticket = 1;
    uint32_t max_queued = 0;
    bool stop = false;
    std::thread th;
    uint64_t n_done = 0, n_failed = 0, n_cancelled = 0;
    // graphs, timing, concurrent, long item: restored at destroy
    int64_t saved_opts[4] = {0, 0, 1, -2};
    std::atomic<int> running{0};  // admitted requests not yet completed
};

namespace {

struct CbArg {
    logan_server* s;
    uint64_t ticket;
    const void* staged_results;  // null: results were copied directly
    void* results;
    size_t result_bytes;
};

// host callback at the end of a request's stream work: no CUDA calls here
void CUDART_CB on_done(void* p) {
    CbArg* a = static_cast<CbArg*>(p);
    logan_server* s = a->s;
    if (a->staged_results) std::memcpy(a->results, a->staged_results, a->result_bytes);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->reqs.find(a->ticket);
        if (it != s->reqs.end()) {
            Req& q = it->second;
            q.state = St::Done;
            q.t_done = now_s();
            s->arena.release(q.off, q.bytes);
            if (q.hbytes) s->harena.release(q.hoff, q.hbytes);
            s->slots[q.slot].ticket = 0;
            s->running.fetch_sub(1);
            s->n_done++;
        }
    }
    s->cv.notify_all();
    s->done_cv.notify_all();
    delete a;
}

// Enqueue one admitted request on its slot's stream.  Called without the lock.
int launch(logan_server* s, uint64_t ticket, Req& q) {
    cudaStream_t st = s->slots[q.slot].stream;
    char* base = s->dev + q.off;
    size_t at = 0;
    auto place = [&](size_t n) {
        char* p = base + at;
        at += up(n);
        return p;
    };
    const logan_request_t& r = q.r;
    // host source of each copy: the pinned staging area (filled here) or,
    // for a request too large for it, the caller's buffer itself
    char* hbase = q.hbytes ? s->host + q.hoff : nullptr;
    size_t hat = 0;
    auto h2d = [&](void* dst, const void* src, size_t n) -> cudaError_t {
        if (!n) return cudaSuccess;
        const void* from = src;
        if (hbase) {
            char* h = hbase + hat;
            hat += up(n);
            std::memcpy(h, src, n);
            from = h;
        }
        return cudaMemcpyAsync(dst, from, n, cudaMemcpyHostToDevice, st);
    };
    auto copy_pool = [&](const logan_seqs_t& h, logan_seqs_t& d) -> cudaError_t {
        const size_t nb = h.packed2bit ? ((h.pool_bases + 15) / 16 + 1) * 4 : h.pool_bases;
        char* b = place(nb);
        char* o = place(size_t(h.count) * 8);
        char* l = place(size_t(h.count) * 4);
        cudaError_t e = cudaSuccess;
        if (nb && h.bases) {
            // the spare word of a packed pool is zeroed here
            const size_t have = pool_host_bytes(h);
            e = h2d(b, h.bases, have);
            if (e == cudaSuccess && nb > have) e = cudaMemsetAsync(b + have, 0, nb - have, st);
        }
        if (e == cudaSuccess && h.count) e = h2d(o, h.offsets, size_t(h.count) * 8);
        if (e == cudaSuccess && h.count) e = h2d(l, h.lengths, size_t(h.count) * 4);
        d = h;
        d.bases = b;
        d.offsets = reinterpret_cast<const uint64_t*>(o);
        d.lengths = reinterpret_cast<const uint32_t*>(l);
        return e;
    };
    logan_seqs_t dA, dB;
    cudaError_t e = copy_pool(r.A, dA);
    if (e == cudaSuccess) {
        if (r.same_pool) dB = dA;
        else e = copy_pool(r.B, dB);
    }
    char* seeds = place(size_t(r.n_pairs) * sizeof(logan_seed_t));
    char* xs = r.X_per_pair ? place(size_t(r.n_pairs) * 4) : nullptr;
    char* res = place(size_t(r.n_pairs) * sizeof(logan_result_t));
    char* ws = place(q.ws_bytes);
    if (e == cudaSuccess) e = h2d(seeds, r.seeds, size_t(r.n_pairs) * sizeof(logan_seed_t));
    if (e == cudaSuccess && xs) e = h2d(xs, r.X_per_pair, size_t(r.n_pairs) * 4);
    if (e != cudaSuccess) return LOGAN_ECUDA;
    // with the GPU nearly idle, long extensions run one to a warp (shorter
    // latency); with several requests in flight every extension runs in the
    // several-to-a-warp forms (more extensions per instruction)
    logan_set_option(s->ctx, LOGAN_OPT_LONG_ITEM, s->running.load() <= 8 ? 65536 : -1);
    int rc = logan_extend_batch(s->ctx, &dA, &dB, reinterpret_cast<const logan_seed_t*>(seeds),
                                r.n_pairs, r.match, r.mismatch, r.gap, r.X,
                                reinterpret_cast<const int32_t*>(xs), ws, q.ws_bytes,
                                reinterpret_cast<logan_result_t*>(res), st);
    if (rc != LOGAN_OK) return rc;
    const size_t rbytes = size_t(r.n_pairs) * sizeof(logan_result_t);
    void* hres = hbase ? static_cast<void*>(hbase + hat) : static_cast<void*>(r.results);
    e = cudaMemcpyAsync(hres, res, rbytes, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return LOGAN_ECUDA;
    CbArg* a = new CbArg{s, ticket, hbase ? hres : nullptr, r.results, rbytes};
    if (cudaLaunchHostFunc(st, on_done, a) != cudaSuccess) {
        delete a;
        return LOGAN_ECUDA;
    }
    return LOGAN_OK;
}

void scheduler(logan_server* s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        // admit in arrival order while a slot is idle and the arena has room
        bool progressed = false;
        while (!s->queue.empty()) {
            const uint64_t t = s->queue.front();
            auto it = s->reqs.find(t);
            if (it == s->reqs.end() || it->second.state != St::Queued) {
                s->queue.pop_front();
                continue;
            }
            Req& q = it->second;
            int slot = -1;
            for (size_t k = 0; k < s->slots.size(); ++k)
                if (s->slots[k].ticket == 0) {
                    slot = int(k);
                    break;
                }
            size_t off = 0, hoff = 0;
            if (slot < 0 || !s->arena.alloc(q.bytes, &off)) break;
            if (q.hbytes && !s->harena.alloc(q.hbytes, &hoff)) {
                s->arena.release(off, q.bytes);
                break;
            }
            q.hoff = hoff;
            s->queue.pop_front();
            q.state = St::Running;
            q.slot = slot;
            q.off = off;
            q.t_admit = now_s();
            s->slots[slot].ticket = t;
            s->running.fetch_add(1);
            lk.unlock();
            const int rc = launch(s, t, q);  // q stays valid: entries are erased only when done
            lk.lock();
            if (rc != LOGAN_OK) {
                // nothing of this request will complete on the device; wait for
                // whatever was enqueued, then return its memory
                lk.unlock();
                cudaStreamSynchronize(s->slots[slot].stream);
                lk.lock();
                q.state = St::Failed;
                q.status = rc;
                q.t_done = now_s();
                s->arena.release(q.off, q.bytes);
                if (q.hbytes) s->harena.release(q.hoff, q.hbytes);
                s->slots[slot].ticket = 0;
                s->running.fetch_sub(1);
                s->n_failed++;
                s->done_cv.notify_all();
            }
            progressed = true;
        }
        if (s->stop) {
            bool busy = false;
            for (auto& sl : s->slots) busy |= sl.ticket != 0;
            if (!busy) break;
        }
        if (!progressed) s->cv.wait(lk);
    }
}

}  // namespace

extern "C" {

int logan_server_create(logan_ctx_t* ctx, size_t budget_bytes, int max_inflight,
                        uint32_t max_queued, logan_server_t** out) {
    if (!ctx || !out || budget_bytes == 0 || max_inflight < 1 || max_inflight > 64)
        return LOGAN_EINVAL;
    *out = nullptr;
    int64_t dev = 0;
    if (logan_get_option(ctx, LOGAN_OPT_DEVICE, &dev) != LOGAN_OK) return LOGAN_EINVAL;
    logan_server* s = new (std::nothrow) logan_server();
    if (!s) return LOGAN_ENOMEM;
    s->ctx = ctx;
    s->device = int(dev);
    s->max_queued = max_queued ? max_queued : 1u << 20;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(s->device);
    int rc = LOGAN_OK;
    if (cudaMalloc(&s->dev, budget_bytes) != cudaSuccess) rc = LOGAN_ENOMEM;
    const size_t hsize = staging_bytes(budget_bytes);
    if (rc == LOGAN_OK && cudaHostAlloc(reinterpret_cast<void**>(&s->host), hsize,
                                        cudaHostAllocDefault) != cudaSuccess)
        rc = LOGAN_ENOMEM;
    s->slots.resize(size_t(max_inflight));
    for (auto& sl : s->slots)
        if (rc == LOGAN_OK && cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess)
            rc = LOGAN_ECUDA;
    cudaSetDevice(prev);
    if (rc != LOGAN_OK) {
        for (auto& sl : s->slots)
            if (sl.stream) cudaStreamDestroy(sl.stream);
        if (s->dev) cudaFree(s->dev);
        if (s->host) cudaFreeHost(s->host);
        delete s;
        return rc;
    }
    s->arena.init(budget_bytes);
    s->harena.init(hsize);
    // the scheduler owns the context from now on: graphs off (every request
    // has its own pointers), no timing, and every request's levels on its
    // slot stream (requests already overlap across slots; more streams per
    // request would only share the device's hardware queues, so that a long
    // extension in one request could hold back another request's launches)
    logan_get_option(ctx, LOGAN_OPT_GRAPHS, &s->saved_opts[0]);
    logan_get_option(ctx, LOGAN_OPT_TIMING, &s->saved_opts[1]);
    logan_get_option(ctx, LOGAN_OPT_CONCURRENT, &s->saved_opts[2]);
    logan_get_option(ctx, LOGAN_OPT_LONG_ITEM, &s->saved_opts[3]);
    logan_set_option(ctx, LOGAN_OPT_GRAPHS, 0);
    logan_set_option(ctx, LOGAN_OPT_TIMING, 0);
    logan_set_option(ctx, LOGAN_OPT_CONCURRENT, 0);
    // a request is small next to the GPU but shares it with the other
    // slots: the scheduler picks LOGAN_OPT_LONG_ITEM per request from the
    // load (the automatic rule would put every item of a small request in
    // the latency forms)
    logan_set_option(ctx, LOGAN_OPT_LONG_ITEM, 65536);
    s->th = std::thread(scheduler, s);
    *out = s;
    return LOGAN_OK;
}

int logan_server_submit(logan_server_t* s, const logan_request_t* r, uint64_t* ticket) {
    if (!s || !r || !ticket) return LOGAN_EINVAL;
    if (r->n_pairs == 0 || !r->seeds || !r->results) return LOGAN_EINVAL;
    const logan_seqs_t& B = r->same_pool ? r->A : r->B;
    size_t ws = 0;
    int rc = logan_workspace_size(s->ctx, &r->A, &B, r->n_pairs, &ws);
    if (rc != LOGAN_OK) return rc;
    size_t bytes = pool_bytes(r->A) + (r->same_pool ? 0 : pool_bytes(r->B)) +
                   up(size_t(r->n_pairs) * sizeof(logan_seed_t)) +
                   (r->X_per_pair ? up(size_t(r->n_pairs) * 4) : 0) +
                   up(size_t(r->n_pairs) * sizeof(logan_result_t)) + up(ws);
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return LOGAN_ECANCELED;
    if (bytes > s->arena.size()) return LOGAN_ENOMEM;        // can never fit
    if (s->queue.size() >= s->max_queued) return LOGAN_EAGAIN;  // back-pressure
    const uint64_t t = s->next_ticket++;
    Req q;
    q.r = *r;
    if (r->same_pool) q.r.B = r->A;
    q.bytes = bytes;
    q.ws_bytes = ws;
    const size_t hb = request_host_bytes(q.r);
    q.hbytes = (hb <= s->harena.size() && !request_pinned(q.r)) ? hb : 0;
    q.t_submit = now_s();
    s->reqs.emplace(t, q);
    s->queue.push_back(t);
    *ticket = t;
    s->cv.notify_all();
    return LOGAN_OK;
}

static int finish(logan_server* s, std::unordered_map<uint64_t, Req>::iterator it, int* status,
                  double* latency_ms) {
    Req& q = it->second;
    if (status) *status = q.state == St::Cancelled ? LOGAN_ECANCELED : q.status;
    if (latency_ms) *latency_ms = (q.t_done - q.t_submit) * 1e3;
    s->reqs.erase(it);
    return LOGAN_OK;
}

int logan_server_poll(logan_server_t* s, uint64_t ticket, int* done, int* status,
                      double* latency_ms) {
    if (!s || !done) return LOGAN_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return LOGAN_ENOTFOUND;
    const St st = it->second.state;
    *done = (st == St::Done || st == St::Failed || st == St::Cancelled) ? 1 : 0;
    if (!*done) return LOGAN_OK;
    return finish(s, it, status, latency_ms);
}

int logan_server_wait(logan_server_t* s, uint64_t ticket, int timeout_ms, int* status,
                      double* latency_ms) {
    if (!s) return LOGAN_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto ready = [&] {
        auto it = s->reqs.find(ticket);
        if (it == s->reqs.end()) return true;
        const St st = it->second.state;
        return st == St::Done || st == St::Failed || st == St::Cancelled;
    };
    if (timeout_ms < 0) s->done_cv.wait(lk, ready);
    else if (!s->done_cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready))
        return LOGAN_ETIMEOUT;
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return LOGAN_ENOTFOUND;
    return finish(s, it, status, latency_ms);
}

int logan_server_cancel(logan_server_t* s, uint64_t ticket) {
    if (!s) return LOGAN_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return LOGAN_ENOTFOUND;
    Req& q = it->second;
    if (q.state != St::Queued) return LOGAN_EAGAIN;  // admitted: runs to completion
    q.state = St::Cancelled;
    q.t_done = now_s();
    s->n_cancelled++;
    s->done_cv.notify_all();
    return LOGAN_OK;
}

int logan_server_stats(logan_server_t* s, logan_server_stats_t* out) {
    if (!s || !out) return LOGAN_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    out->queued = uint32_t(s->queue.size());
    uint32_t running = 0;
    for (auto& sl : s->slots) running += sl.ticket != 0;
    out->running = running;
    out->completed = s->n_done;
    out->failed = s->n_failed;
    out->cancelled = s->n_cancelled;
    out->budget_bytes = s->arena.size();
    out->used_bytes = s->arena.used();
    out->peak_bytes = s->arena.peak();
    return LOGAN_OK;
}

int logan_server_destroy(logan_server_t* s) {
    if (!s) return LOGAN_EINVAL;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        // queued requests will never run
        for (uint64_t t : s->queue) {
            auto it = s->reqs.find(t);
            if (it != s->reqs.end() && it->second.state == St::Queued) it->second.state = St::Cancelled;
        }
        s->queue.clear();
    }
    s->cv.notify_all();
    s->done_cv.notify_all();
    if (s->th.joinable()) s->th.join();  // returns once running requests completed
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(s->device);
    for (auto& sl : s->slots) {
        if (sl.stream) {
            cudaStreamSynchronize(sl.stream);
            cudaStreamDestroy(sl.stream);
        }
    }
    cudaFree(s->dev);
    cudaFreeHost(s->host);
    cudaSetDevice(prev);
    logan_set_option(s->ctx, LOGAN_OPT_GRAPHS, s->saved_opts[0]);
    logan_set_option(s->ctx, LOGAN_OPT_TIMING, s->saved_opts[1]);
    logan_set_option(s->ctx, LOGAN_OPT_CONCURRENT, s->saved_opts[2]);
    logan_set_option(s->ctx, LOGAN_OPT_LONG_ITEM, s->saved_opts[3]);
    delete s;
    return LOGAN_OK;
}

}  // extern "C"
