// Serving loop: blocks arrive one by one as reconciliation emits them
// (Sec. 2.2: each reconciled block X is compressed to Y = g(X)), are admitted
// while their device footprint fits a budget, and run as continuously formed
// batches that overlap on several device streams. Host-side only; the hashing
// itself is pa_hash_batched (pa_hash for a batch of one).
//
// Worker thread, one pass of its loop:
//   1. in-flight batches whose completion event has been reached release
//      their footprint and complete their tickets (with the status of their
//      stream's status word, read behind the batch);
//   2. while a stream slot is free and the head of the FIFO fits in the
//      budget, requests are taken (up to max_batch) and queued as one batch,
//      followed by the status-word read and the completion event;
//   3. with nothing done in the pass it yields and polls again, or, once
//      nothing has happened for idle_poll_us and no batch is in flight, sleeps
//      on a condition variable until pa_submit (or pa_serve_stop) wakes it.
// Polling the events instead of a host callback plus a wake-up keeps the
// completion latency at the polling interval (microseconds).
// pa_poll waits on a second condition variable, notified when tickets complete.
#include <stdlib.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/pa.h"
#include "pa_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t ticket;
    pa_block blk;
    uint64_t footprint;
    Clock::time_point t_submit;
};

struct Batch {
    std::vector<Request> reqs;
    uint64_t footprint = 0;
    int slot = -1;
    const volatile uint32_t* status = nullptr;  // the stream's status word, copied behind the batch
};

struct Result {
    bool done = false;
    int status = PA_OK;
};

struct Server {
    std::mutex mu;
    std::condition_variable wake;      // the worker: a submission or a stop
    std::condition_variable done_cv;   // pa_poll: tickets completed
    bool running = false, stopping = false;
    int device = 0;
    pa_config cfg{};
    std::thread worker;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> events;    // per stream: recorded behind its batch
    std::vector<Batch*> slot_busy;      // per stream: batch in flight or null
    std::deque<Request> pending;
    std::unordered_map<uint64_t, Result> results;
    uint64_t next_ticket = 1;
    uint64_t inflight_bytes = 0;
    // statistics
    uint64_t completed = 0, bits_done = 0, batches = 0, peak_bytes = 0, peak_inflight = 0;
    std::vector<double> latency_us;
    Clock::time_point t_first, t_last;
};

Server g_srv;

uint64_t footprint_of(const pa_block& b) {
    uint64_t io = 3 * ((b.n + 63) / 64) * 8 + ((b.m + 63) / 64) * 8;
    return pa_workspace_bytes(b.n) + io;
}

void finish_batch(Batch* b, int status, Clock::time_point t) {  // with g_srv.mu held
    for (const Request& r : b->reqs) {
        Result& res = g_srv.results[r.ticket];
        res.done = true;
        res.status = status;
        g_srv.completed++;
        g_srv.bits_done += r.blk.n;
        g_srv.latency_us.push_back(std::chrono::duration<double, std::micro>(t - r.t_submit).count());
    }
    g_srv.t_last = t;
    g_srv.inflight_bytes -= b->footprint;
    if (b->slot >= 0) g_srv.slot_busy[b->slot] = nullptr;
    delete b;
    g_srv.done_cv.notify_all();
}

// 1. retire: batches whose event has been reached; true if any was
bool retire_locked() {
    bool any = false;
    for (size_t s = 0; s < g_srv.slot_busy.size(); s++) {
        Batch* b = g_srv.slot_busy[s];
        if (!b) continue;
        cudaError_t q = cudaEventQuery(g_srv.events[s]);
        if (q == cudaErrorNotReady) continue;
        int st = PA_OK;
        if (q != cudaSuccess) st = PA_ECUDA;
        else if (b->status && (*b->status & pa::PA_STATUS_TIMEOUT)) st = PA_ETIMEOUT;
        finish_batch(b, st, Clock::now());
        any = true;
    }
    return any;
}

// 2. admit one batch into a free slot; true if one was queued
bool admit_locked(std::unique_lock<std::mutex>& lk) {
    int slot = -1;
    for (size_t s = 0; s < g_srv.slot_busy.size(); s++)
        if (!g_srv.slot_busy[s]) { slot = (int)s; break; }
    if (slot < 0 || g_srv.pending.empty()) return false;
    Batch* b = new Batch;
    b->slot = slot;
    while (!g_srv.pending.empty() && b->reqs.size() < g_srv.cfg.max_batch) {
        const Request& r = g_srv.pending.front();
        if (g_srv.inflight_bytes + b->footprint + r.footprint > g_srv.cfg.hbm_budget_bytes) break;
        b->footprint += r.footprint;
        b->reqs.push_back(r);
        g_srv.pending.pop_front();
    }
    if (b->reqs.empty()) {  // the head of the line waits for memory to free up
        delete b;
        return false;
    }
    g_srv.inflight_bytes += b->footprint;
    g_srv.peak_bytes = std::max(g_srv.peak_bytes, g_srv.inflight_bytes);
    g_srv.slot_busy[slot] = b;
    g_srv.batches++;
    uint64_t n_inflight = 0;
    for (Batch* x : g_srv.slot_busy) n_inflight += x ? x->reqs.size() : 0;
    g_srv.peak_inflight = std::max(g_srv.peak_inflight, n_inflight);
    std::vector<pa_block> blocks;
    for (const Request& r : b->reqs) blocks.push_back(r.blk);
    cudaStream_t st = g_srv.streams[slot];
    cudaEvent_t ev = g_srv.events[slot];
    lk.unlock();  // queueing takes the library lock; do not hold ours
    // a lone request takes the single-block path (no side-stream fork)
    const pa_block& b0 = blocks[0];
    int rc = blocks.size() == 1 ? pa_hash(b0.key, b0.seed_a, b0.seed_b, b0.n, b0.m, b0.out, st)
                                : pa_hash_batched(blocks.data(), (uint32_t)blocks.size(), st);
    const volatile uint32_t* word = nullptr;
    if (rc == PA_OK) rc = pa::queue_status_read(st, true, &word);
    cudaError_t e = rc == PA_OK ? cudaEventRecord(ev, st) : cudaSuccess;
    lk.lock();
    b->status = word;
    if (rc != PA_OK || e != cudaSuccess) finish_batch(b, rc != PA_OK ? rc : PA_ECUDA, Clock::now());
    return true;
}

void worker_main() {
    cudaSetDevice(g_srv.device);
    std::unique_lock<std::mutex> lk(g_srv.mu);
    Clock::time_point last_event = Clock::now();
    const auto idle = std::chrono::microseconds(g_srv.cfg.idle_poll_us);
    while (true) {
        bool progress = retire_locked();
        if (g_srv.stopping && g_srv.pending.empty()) {
            bool idle_now = true;
            for (Batch* b : g_srv.slot_busy) idle_now = idle_now && !b;
            if (idle_now) break;
        }
        while (admit_locked(lk)) progress = true;
        if (progress) {
            last_event = Clock::now();
            continue;
        }
        bool inflight = false;
        for (Batch* b : g_srv.slot_busy) inflight = inflight || b;
        if (inflight || g_srv.cfg.idle_poll_us == 0 || Clock::now() - last_event < idle) {
            // poll: completions and submissions are expected soon
            lk.unlock();
            std::this_thread::yield();
            lk.lock();
            continue;
        }
        // nothing in flight for a while: sleep until a submission (or a stop)
        g_srv.wake.wait(lk, [] { return !g_srv.pending.empty() || g_srv.stopping; });
        last_event = Clock::now();
    }
}

int start_locked(int device, const pa_config* cfg) {
    if (g_srv.running) return PA_OK;
    int dev = 0;
    if (device >= 0) {
        if (cudaSetDevice(device) != cudaSuccess) {
            cudaGetLastError();
            return PA_EINVAL;
        }
    }
    if (cudaGetDevice(&dev) != cudaSuccess) return PA_ECUDA;
    g_srv.device = dev;
    pa_config c{};
    if (cfg) c = *cfg;
    if (!c.max_batch || c.max_batch > 1024) c.max_batch = 64;
    if (!c.streams || c.streams > 8) c.streams = 2;
    if (!c.max_pending) c.max_pending = 1u << 16;
    if (!c.hbm_budget_bytes) {
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return PA_ECUDA;
        c.hbm_budget_bytes = free_b / 2;
    }
    g_srv.cfg = c;
    g_srv.streams.assign(c.streams, nullptr);
    g_srv.events.assign(c.streams, nullptr);
    for (uint32_t i = 0; i < c.streams; i++)
        if (cudaStreamCreateWithFlags(&g_srv.streams[i], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&g_srv.events[i], cudaEventDisableTiming) != cudaSuccess)
            return PA_ECUDA;
    g_srv.slot_busy.assign(c.streams, nullptr);
    g_srv.stopping = false;
    g_srv.running = true;
    g_srv.worker = std::thread(worker_main);
    return PA_OK;
}

}  // namespace

extern "C" {

int pa_init(int device, const pa_config* cfg) {
    std::lock_guard<std::mutex> lk(g_srv.mu);
    if (g_srv.running) {
        pa::set_error("pa_init: serving loop already running");
        return PA_EINVAL;
    }
    int rc = start_locked(device, cfg);
    if (rc == PA_EINVAL) pa::set_error("pa_init: not a valid CUDA device");
    else if (rc) pa::set_error("pa_init: CUDA set-up failed");
    return rc;
}

int pa_submit(const pa_block* blk, uint64_t* ticket) {
    if (!blk || !ticket || !blk->key || !blk->seed_a || !blk->seed_b || !blk->out) {
        pa::set_error("pa_submit: null pointer");
        return PA_EINVAL;
    }
    if (blk->n < 1 || blk->m < 1 || blk->m > blk->n || blk->n > PA_MAX_BITS) {
        pa::set_error("pa_submit: need 1 <= m <= n <= PA_MAX_BITS");
        return PA_EINVAL;
    }
    std::lock_guard<std::mutex> lk(g_srv.mu);
    int rc = start_locked(-1, nullptr);
    if (rc) {
        pa::set_error("pa_submit: CUDA set-up failed");
        return rc;
    }
    uint64_t fp = footprint_of(*blk);
    if (fp > g_srv.cfg.hbm_budget_bytes) {
        pa::set_error("pa_submit: block footprint exceeds the HBM budget");
        return PA_EINVAL;
    }
    if (g_srv.pending.size() >= g_srv.cfg.max_pending) {
        pa::set_error("pa_submit: queue full");
        return PA_EAGAIN;
    }
    Request r{g_srv.next_ticket++, *blk, fp, Clock::now()};
    if (g_srv.completed == 0 && g_srv.pending.empty() && g_srv.batches == 0) g_srv.t_first = r.t_submit;
    g_srv.results[r.ticket] = Result{};
    g_srv.pending.push_back(r);
    *ticket = r.ticket;
    g_srv.wake.notify_one();
    return PA_OK;
}

int pa_poll(uint64_t ticket, uint32_t timeout_us, int* status) {
    std::unique_lock<std::mutex> lk(g_srv.mu);
    auto it = g_srv.results.find(ticket);
    if (it == g_srv.results.end()) {
        pa::set_error("pa_poll: unknown ticket");
        return PA_EINVAL;
    }
    auto deadline = Clock::now() + std::chrono::microseconds(timeout_us);
    while (!it->second.done) {
        if (g_srv.done_cv.wait_until(lk, deadline) == std::cv_status::timeout) break;
        it = g_srv.results.find(ticket);
    }
    if (!it->second.done) return PA_EAGAIN;
    if (status) *status = it->second.status;
    g_srv.results.erase(it);
    return PA_OK;
}

int pa_serve_stats(pa_serve_stats_t* out) {
    if (!out) return PA_EINVAL;
    std::lock_guard<std::mutex> lk(g_srv.mu);
    pa_serve_stats_t s{};
    s.completed = g_srv.completed;
    s.pending = g_srv.pending.size();
    s.batches = g_srv.batches;
    s.bits = g_srv.bits_done;
    s.peak_inflight_bytes = g_srv.peak_bytes;
    s.peak_inflight_blocks = g_srv.peak_inflight;
    s.hbm_budget_bytes = g_srv.cfg.hbm_budget_bytes;
    if (!g_srv.latency_us.empty()) {
        std::vector<double> v = g_srv.latency_us;
        std::sort(v.begin(), v.end());
        auto pct = [&](double q) { return v[std::min(v.size() - 1, (size_t)(q * (v.size() - 1) + 0.5))]; };
        s.p50_us = pct(0.50);
        s.p99_us = pct(0.99);
        s.max_us = v.back();
        double span = std::chrono::duration<double>(g_srv.t_last - g_srv.t_first).count();
        s.mbps = span > 0 ? g_srv.bits_done / span / 1e6 : 0;
    }
    *out = s;
    return PA_OK;
}

int pa_serve_stop(void) {
    std::thread w;
    {
        std::lock_guard<std::mutex> lk(g_srv.mu);
        if (!g_srv.running) return PA_OK;
        g_srv.stopping = true;
        g_srv.wake.notify_all();
        w = std::move(g_srv.worker);
    }
    w.join();
    std::lock_guard<std::mutex> lk(g_srv.mu);
    for (auto s : g_srv.streams) cudaStreamDestroy(s);
    for (auto e : g_srv.events) cudaEventDestroy(e);
    g_srv.streams.clear();
    g_srv.events.clear();
    g_srv.slot_busy.clear();
    g_srv.running = false;
    g_srv.completed = g_srv.bits_done = g_srv.batches = g_srv.peak_bytes = g_srv.peak_inflight = 0;
    g_srv.latency_us.clear();
    return PA_OK;
}

}  // extern "C"
