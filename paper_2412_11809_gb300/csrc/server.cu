// Serving loop: many detector streams on one GPU under one device-memory
// budget, with admission as memory frees up (continuous batching of chunks).
//
// The paper's pipeline keeps every buffer "in use until retrieved" and lets a
// thread take the next buffer only when one is free (Algorithm 2, and
// Algorithm 3 steps 1 and 9, Section 4.1).  Here the unit is a chunk of one
// detector stream: a submitted chunk waits in one queue, in submission
// order, until its stream is idle and the device memory it needs fits in the
// budget; then its stream's worker thread pushes it into the stream's
// streaming context (open clusters carried on the device, finalised by the
// ToA watermark) on the stream's own CUDA stream and copies the finalised
// labels, their global indices and records into the caller's host buffers.
// Chunks of different streams run concurrently and overlap on the GPU.
//
// Memory.  A stream holds its carry buffers all the time and its work
// arrays and outputs while a chunk is in flight.  Admission reserves what the
// context will hold once the chunk has run (ctx_projected_bytes); when the
// result is in the caller's buffers the reservation becomes the context's
// actual holding.  When the chunk at the head of the queue does not fit, the
// work arrays of idle streams are dropped (stream-ordered frees, no device
// synchronisation) before it waits; chunks behind it do not overtake it
// (no starvation of large chunks).  A chunk that cannot fit even in an
// otherwise empty budget completes at once with TPC_ERR_BUSY.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "ctx_internal.h"
#include "tpc_internal.cuh"

using namespace tpc;
using Clock = std::chrono::steady_clock;

namespace {

struct Request {
    int stream = 0;
    const tpc_hit *hits = nullptr;
    size_t n = 0;
    uint64_t *labels = nullptr, *indices = nullptr;
    tpc_cluster *records = nullptr;
    size_t cap = 0;
    uint64_t tag = 0;
    bool end = false;          // end of stream: close every open cluster
    Clock::time_point t_submit, t_admit;
    size_t reserve = 0;        // bytes reserved at admission
    bool waited = false;       // has waited for memory at the head of the queue
};

struct Stream {
    tpc_ctx *ctx = nullptr;
    bool busy = false;         // a chunk is admitted and not yet completed
    bool ended = false;        // an end-of-stream chunk was submitted
    size_t held = 0;           // bytes the context holds while idle
    std::unique_ptr<Request> job;
    std::condition_variable cv;
    std::thread worker;
};

double ms_between(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
}

}  // namespace

static_assert(sizeof(tpc_server_result) == 48, "result layout");
static_assert(sizeof(tpc_server_stats) == 13 * 8, "stats layout");

struct tpc_server {
    uint64_t budget = 0;
    std::mutex mu;
    std::condition_variable done_cv;
    std::deque<std::unique_ptr<Request>> pending;
    std::deque<tpc_server_result> done;
    std::vector<std::unique_ptr<Stream>> streams;
    uint64_t in_use = 0;       // sum of idle holdings and admitted reservations
    tpc_server_stats st{};
    bool stopping = false;
    int device = 0;

    // Admit what fits, in submission order (call with mu held).
    void admit() {
        for (auto it = pending.begin(); it != pending.end();) {
            Request &r = **it;
            Stream &s = *streams[r.stream];
            if (s.busy) { ++it; continue; }   // its stream's earlier chunk is still running
            const size_t proj = ctx_projected_bytes(s.ctx, r.end ? 0 : r.n);
            const uint64_t others = in_use - s.held;
            if (proj > budget) {   // never fits: complete it with an error
                finish_now(r, TPC_ERR_BUSY);
                it = pending.erase(it);
                continue;
            }
            if (others + proj > budget) {
                // make room: drop the work arrays of idle streams (their carry stays)
                for (auto &o : streams) {
                    if (o->busy || o.get() == &s) continue;
                    const size_t before = o->held;
                    ctx_release_scratch(o->ctx);
                    o->held = ctx_held_bytes(o->ctx);
                    in_use -= before - o->held;
                    if (o->held != before) ++st.releases;
                    if (in_use - s.held + proj <= budget) break;
                }
            }
            if (in_use - s.held + proj > budget) {
                bool running = false;
                for (const auto &o : streams) running = running || o->busy;
                if (!running) {   // nothing will free memory: the carry of the other streams is too big
                    finish_now(r, TPC_ERR_BUSY);
                    it = pending.erase(it);
                    continue;
                }
                if (!r.waited) ++st.waits;
                r.waited = true;
                break;   // the head waits; later chunks do not overtake it
            }
            in_use = in_use - s.held + proj;
            if (in_use > st.peak) st.peak = in_use;
            r.reserve = proj;
            r.t_admit = Clock::now();
            s.busy = true;
            s.job = std::move(*it);
            it = pending.erase(it);
            ++st.admitted;
            s.cv.notify_one();
        }
    }

    void finish_now(const Request &r, int status) {
        tpc_server_result res{};
        res.tag = r.tag;
        res.stream = r.stream;
        res.status = status;
        res.latency_ms = ms_between(r.t_submit, Clock::now());
        done.push_back(res);
        ++st.completed;
        ++st.rejected;
        done_cv.notify_all();
    }

    // The worker of stream k: runs its admitted chunks one after another.
    void work(int k) {
        Stream &s = *streams[k];
        if (cudaSetDevice(device) != cudaSuccess) return;
        std::unique_lock<std::mutex> lk(mu);
        while (true) {
            s.cv.wait(lk, [&] { return stopping || s.job; });
            if (!s.job) return;   // stopping
            std::unique_ptr<Request> r = std::move(s.job);
            lk.unlock();
            tpc_server_result res{};
            res.tag = r->tag;
            res.stream = k;
            int rc = r->end ? tpc_flush(s.ctx) : tpc_push(s.ctx, r->hits, r->n, TPC_HOST);
            size_t n_out = 0, n_rec = 0;
            if (rc == TPC_OK) rc = tpc_labels(s.ctx, r->labels, r->indices, r->cap, &n_out, TPC_HOST);
            if (rc == TPC_OK) rc = tpc_cluster_features(s.ctx, r->records, r->cap, &n_rec, TPC_HOST);
            if (rc == TPC_OK) rc = ctx_settle(s.ctx);   // exact carry: the next projection is tight
            const size_t held = ctx_held_bytes(s.ctx);
            const Clock::time_point t_done = Clock::now();
            res.status = rc;
            res.n_hits = n_out;
            res.n_clusters = n_rec;
            res.queue_ms = ms_between(r->t_submit, r->t_admit);
            res.latency_ms = ms_between(r->t_submit, t_done);
            lk.lock();
            in_use = in_use - r->reserve + held;
            s.held = held;
            s.busy = false;
            done.push_back(res);
            ++st.completed;
            if (rc != TPC_OK) ++st.failed;
            done_cv.notify_all();
            admit();
        }
    }
};

extern "C" {

int tpc_server_create(uint64_t mem_budget, tpc_server **out) {
    if (!out) return TPC_ERR_ARG;
    *out = nullptr;
    if (mem_budget == 0) return TPC_ERR_ARG;
    tpc_server *s = new (std::nothrow) tpc_server();
    if (!s) return TPC_ERR_NOMEM;
    if (cudaGetDevice(&s->device) != cudaSuccess) { delete s; return TPC_ERR_CUDA; }
    s->budget = mem_budget;
    s->st.budget = mem_budget;
    *out = s;
    return TPC_OK;
}

int tpc_server_add_stream(tpc_server *s, uint32_t width, uint32_t height, uint64_t dt,
                          uint64_t max_disorder, int *id) {
    if (!s || !id || max_disorder == 0 || max_disorder == ~0ull) return TPC_ERR_ARG;
    tpc_ctx *c = nullptr;
    int rc = tpc_create(width, height, dt, TPC_LOCAL, &c);
    if (rc) return rc;
    rc = tpc_set_option(c, TPC_OPT_MAX_DISORDER, max_disorder);
    if (rc) { tpc_destroy(c); return rc; }
    std::unique_ptr<Stream> st(new (std::nothrow) Stream());
    if (!st) { tpc_destroy(c); return TPC_ERR_NOMEM; }
    st->ctx = c;
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stopping) { tpc_destroy(c); return TPC_ERR_STATE; }
    st->held = ctx_held_bytes(c);
    s->in_use += st->held;
    const int k = (int)s->streams.size();
    s->streams.push_back(std::move(st));
    try {
        s->streams[k]->worker = std::thread(&tpc_server::work, s, k);
    } catch (...) {
        s->in_use -= s->streams[k]->held;
        tpc_destroy(c);
        s->streams.pop_back();
        return TPC_ERR_NOMEM;
    }
    *id = k;
    return TPC_OK;
}

int tpc_server_submit(tpc_server *s, int id, const tpc_hit *hits, size_t n, uint64_t *labels,
                      uint64_t *indices, tpc_cluster *records, size_t cap, uint64_t tag, int end_of_stream) {
    if (!s || (n && !hits) || !labels || !records || (end_of_stream && n)) return TPC_ERR_ARG;
    if (n > 0x7FFFFFFFull) return TPC_ERR_ARG;
    std::unique_ptr<Request> r(new (std::nothrow) Request());
    if (!r) return TPC_ERR_NOMEM;
    r->stream = id;
    r->hits = hits;
    r->n = n;
    r->labels = labels;
    r->indices = indices;
    r->records = records;
    r->cap = cap;
    r->tag = tag;
    r->end = end_of_stream != 0;
    r->t_submit = Clock::now();
    std::lock_guard<std::mutex> lk(s->mu);
    if (id < 0 || id >= (int)s->streams.size()) return TPC_ERR_ARG;
    if (s->stopping || s->streams[id]->ended) return TPC_ERR_STATE;
    if (r->end) s->streams[id]->ended = true;
    s->pending.push_back(std::move(r));
    ++s->st.submitted;
    s->admit();
    return TPC_OK;
}

int tpc_server_wait(tpc_server *s, tpc_server_result *res, int64_t timeout_us) {
    if (!s || !res) return TPC_ERR_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    auto ready = [&] {
        if (!s->done.empty()) return true;
        bool any = !s->pending.empty();
        for (const auto &st : s->streams) any = any || st->busy;
        return !any;   // nothing queued or running: nothing will arrive
    };
    if (timeout_us < 0) s->done_cv.wait(lk, ready);
    else if (!s->done_cv.wait_for(lk, std::chrono::microseconds(timeout_us), ready)) return TPC_ERR_TIMEOUT;
    if (s->done.empty()) return TPC_ERR_STATE;
    *res = s->done.front();
    s->done.pop_front();
    return TPC_OK;
}

int tpc_server_stats_get(tpc_server *s, tpc_server_stats *out) {
    if (!s || !out) return TPC_ERR_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->st;
    out->in_use = s->in_use;
    out->queued = s->pending.size();
    uint64_t busy = 0;
    for (const auto &st : s->streams) busy += st->busy ? 1 : 0;
    out->in_flight = busy;
    out->streams = s->streams.size();
    return TPC_OK;
}

void tpc_server_destroy(tpc_server *s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stopping = true;
        s->pending.clear();   // queued chunks are dropped; running ones finish
        for (auto &st : s->streams) st->cv.notify_all();
    }
    for (auto &st : s->streams) {
        if (st->worker.joinable()) st->worker.join();
        tpc_destroy(st->ctx);
    }
    delete s;
}

}  // extern "C"
