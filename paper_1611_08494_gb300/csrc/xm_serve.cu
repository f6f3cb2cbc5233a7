// xm_serve.cu -- the serving loop: requests against a resident index,
// admitted by device memory and run by continuous batching.
//
// A server owns `slots` host threads, each with its own CUDA stream. A slot
// waits for work, takes the requests at the head of the queue (first come,
// first served) while they fit the batch limits and the unused part of the
// memory budget, runs them as one xm_match_batch on its stream, and marks
// them done. Slots work concurrently: while one batch is on the GPU, the next
// requests to arrive are formed into another batch on another slot, so their
// device work overlaps and nobody waits for a fixed batch boundary. A batch's
// memory stays charged to the budget until all its tickets are released.
// Latency is measured from submission to the moment the batch's results are
// complete on the device (its synchronisation returns).
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "xm_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

// Device bytes a request costs while its batch is in flight and until its
// results are released: keys, prepared sources, per-source results, member
// records, pairs and join rows (about two pairs per source budgeted).
constexpr int64_t kBytesPerA = 480;
constexpr int64_t kBytesPerRequest = 64 << 10;

struct BatchHold {
    xm_batch* batch = nullptr;
    int64_t est = 0;
    int live = 0;  // tickets not yet released
};

struct Ticket {
    int64_t id = 0;
    int state = 0;  // 0 queued, 1 running, 2 done, 3 failed
    xm_status status = XM_OK;
    xm_request req{};
    double* buf = nullptr;  // server-owned device copy of the columns
    int64_t n_a = 0, est = 0;
    Clock::time_point t_submit, t_done;
    std::shared_ptr<BatchHold> hold;
    int64_t index_in_batch = 0;
};

}  // namespace

struct xm_server {
    const xm_index* index = nullptr;
    xm_serve_opts opts{};
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Ticket*> queue;
    std::unordered_map<int64_t, Ticket*> tickets;
    int64_t next_id = 1;
    int64_t mem_in_use = 0, mem_budget = 0;
    bool stopping = false;
    std::vector<std::thread> workers;
    std::vector<cudaStream_t> streams;
    cudaStream_t copy_stream = nullptr;
    // statistics
    int64_t submitted = 0, completed = 0, failed = 0, refused = 0, a_sources = 0, batches = 0;
    std::vector<double> latency_ms;
    int active = 0;
    Clock::time_point busy_since;
    double busy_s = 0.0;
    Clock::time_point window_start;  // latencies of requests submitted before are not kept
};

namespace {

int64_t request_cost(int64_t n_a) { return n_a * kBytesPerA + kBytesPerRequest; }

// The head of the queue fits the unused budget.
bool head_fits(const xm_server* S) {
    return !S->queue.empty() && S->mem_in_use + S->queue.front()->est <= S->mem_budget;
}

void slot_loop(xm_server* S, int k) {
    cudaSetDevice(S->device);
    cudaStream_t st = S->streams[k];
    const xm_serve_opts& o = S->opts;
    for (;;) {
        std::vector<Ticket*> take;
        int64_t est = 0, a_tot = 0;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_work.wait(lk, [&] { return S->stopping || head_fits(S); });
            if (S->stopping) return;
            while (!S->queue.empty()) {
                Ticket* t = S->queue.front();
                if ((int64_t)take.size() >= o.max_batch_requests) break;
                if (!take.empty() && a_tot + t->n_a > o.max_batch_a) break;
                if (S->mem_in_use + est + t->est > S->mem_budget) break;
                S->queue.pop_front();
                t->state = 1;
                take.push_back(t);
                est += t->est;
                a_tot += t->n_a;
            }
            S->mem_in_use += est;
            if (S->active++ == 0) S->busy_since = Clock::now();
        }
        std::vector<xm_request> reqs(take.size());
        for (size_t i = 0; i < take.size(); i++) reqs[i] = take[i]->req;
        xm_batch_opts bo{o.precision, o.use_graph, o.persistent_blocks, 0, 0, 0};
        xm_batch* batch = nullptr;
        const xm_status status =
            xm_match_batch(S->index, reqs.data(), (int64_t)reqs.size(), &bo, st, &batch);
        const Clock::time_point t_done = Clock::now();
        // the inputs are no longer needed once the batch has run
        for (Ticket* t : take) {
            xm::dev_free(t->buf, st);
            t->buf = nullptr;
        }
        {
            std::lock_guard<std::mutex> lk(S->mu);
            auto hold = std::make_shared<BatchHold>();
            hold->batch = batch;
            hold->est = est;
            hold->live = (int)take.size();
            for (size_t i = 0; i < take.size(); i++) {
                Ticket* t = take[i];
                t->status = status;
                t->state = status == XM_OK ? 2 : 3;
                t->t_done = t_done;
                t->hold = hold;
                t->index_in_batch = (int64_t)i;
                if (status == XM_OK) {
                    S->completed++;
                    S->a_sources += t->n_a;
                    if (t->t_submit >= S->window_start)
                        S->latency_ms.push_back(
                            std::chrono::duration<double, std::milli>(t_done - t->t_submit).count());
                } else {
                    S->failed++;
                }
            }
            if (status != XM_OK) {
                // nothing to keep: the budget is returned now
                S->mem_in_use -= est;
                hold->batch = nullptr;
                hold->est = 0;
            }
            S->batches++;
            if (--S->active == 0)
                S->busy_s += std::chrono::duration<double>(Clock::now() - S->busy_since).count();
        }
        S->cv_done.notify_all();
        S->cv_work.notify_all();
    }
}

}  // namespace

using namespace xm;

extern "C" xm_status xm_serve_open(const xm_index* index, const xm_serve_opts* opts, xm_server** out) {
    if (!out || !index) return set_error(XM_EINVAL, "xm_serve_open: bad arguments");
    *out = nullptr;
    xm_server* S = new (std::nothrow) xm_server();
    if (!S) return set_error(XM_ENOMEM, "xm_serve_open: host allocation");
    S->index = index;
    S->window_start = Clock::now();
    if (opts) S->opts = *opts;
    xm_serve_opts& o = S->opts;
    if (o.slots <= 0) o.slots = 2;
    if (o.slots > 16) o.slots = 16;
    if (o.max_batch_requests <= 0) o.max_batch_requests = 256;
    if (o.max_batch_a <= 0) o.max_batch_a = (int64_t)1 << 26;
    if (o.precision != XM_PREC_FP64) o.precision = XM_PREC_FP32_RECHECK;
    cudaGetDevice(&S->device);
    size_t free_b = 0, total_b = 0;
    cudaError_t e = cudaMemGetInfo(&free_b, &total_b);
    if (e != cudaSuccess) {
        delete S;
        return cuda_fail(e, "xm_serve_open: cudaMemGetInfo");
    }
    // blocks the library keeps for reuse are free to the server's own
    // allocations (and go back to the pool when it runs short)
    const double avail = (double)free_b + (double)kept_device_bytes();
    S->mem_budget = o.mem_budget_bytes > 0 ? o.mem_budget_bytes : (int64_t)(0.6 * avail);
    for (int k = 0; k <= o.slots; k++) {
        cudaStream_t st = nullptr;
        e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            for (cudaStream_t q : S->streams) cudaStreamDestroy(q);
            delete S;
            return cuda_fail(e, "xm_serve_open: streams");
        }
        if (k < o.slots) S->streams.push_back(st);
        else S->copy_stream = st;
    }
    for (int k = 0; k < o.slots; k++) S->workers.emplace_back(slot_loop, S, k);
    *out = S;
    return XM_OK;
}

extern "C" xm_status xm_serve_submit(xm_server* S, const xm_request* q, int64_t* ticket) {
    // a request's latency runs from here (its arrival), so the copy of its
    // columns is inside it
    const auto t_arrival = Clock::now();
    if (!S || !q || !ticket) return set_error(XM_EINVAL, "xm_serve_submit: bad arguments");
    *ticket = 0;
    xm_status st = check_request(*q, 0);
    if (st != XM_OK) return st;
    const int64_t n = q->A.n;
    const int64_t est = request_cost(n);
    if (est > S->mem_budget) {
        std::lock_guard<std::mutex> lk(S->mu);
        S->refused++;
        return set_error(XM_EBUSY,
                         "xm_serve_submit: request of %lld A sources needs ~%lld bytes, budget is %lld",
                         (long long)n, (long long)est, (long long)S->mem_budget);
    }
    // copy the columns into server memory so the caller's buffers are free
    Ticket* t = new (std::nothrow) Ticket();
    if (!t) return set_error(XM_ENOMEM, "xm_serve_submit: host allocation");
    t->req = *q;
    t->req.A.id = nullptr;  // A ids are not used by the match
    t->n_a = n;
    t->est = est;
    const double* src[5] = {q->A.lon_deg, q->A.lat_deg, q->region.a_col, q->region.b_col,
                            q->region.pa_col};
    int ncol = 0;
    for (const double* p : src) ncol += p != nullptr;
    if (n > 0) {
        cudaSetDevice(S->device);
        t->buf = (double*)dev_alloc((size_t)ncol * n * sizeof(double), S->copy_stream);
        if (!t->buf) {
            delete t;
            return set_error(XM_ENOMEM, "xm_serve_submit: input copy");
        }
        const double** dst[5] = {&t->req.A.lon_deg, &t->req.A.lat_deg, &t->req.region.a_col,
                                 &t->req.region.b_col, &t->req.region.pa_col};
        int c = 0;
        for (int k = 0; k < 5; k++) {
            if (!src[k]) continue;
            cudaError_t e = cudaMemcpyAsync(t->buf + (int64_t)c * n, src[k], n * sizeof(double),
                                            q->A.on_device ? cudaMemcpyDeviceToDevice
                                                           : cudaMemcpyHostToDevice,
                                            S->copy_stream);
            if (e != cudaSuccess) {
                dev_free(t->buf, S->copy_stream);
                delete t;
                return cuda_fail(e, "xm_serve_submit: input copy");
            }
            *dst[k] = t->buf + (int64_t)c * n;
            c++;
        }
        cudaError_t e = cudaStreamSynchronize(S->copy_stream);
        if (e != cudaSuccess) {
            dev_free(t->buf, S->copy_stream);
            delete t;
            return cuda_fail(e, "xm_serve_submit: input copy");
        }
        t->req.A.on_device = 1;
    }
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->stopping) {
            dev_free(t->buf, S->copy_stream);
            delete t;
            return set_error(XM_EBUSY, "xm_serve_submit: server is closing");
        }
        t->id = S->next_id++;
        t->t_submit = t_arrival;
        S->tickets[t->id] = t;
        S->queue.push_back(t);
        S->submitted++;
        *ticket = t->id;
    }
    S->cv_work.notify_one();
    return XM_OK;
}

extern "C" xm_status xm_serve_poll(xm_server* S, int64_t ticket, int32_t* state) {
    if (!S || !state) return set_error(XM_EINVAL, "xm_serve_poll: bad arguments");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->tickets.find(ticket);
    if (it == S->tickets.end()) return set_error(XM_EINVAL, "xm_serve_poll: unknown ticket");
    *state = it->second->state;
    return XM_OK;
}

extern "C" xm_status xm_serve_wait(xm_server* S, int64_t ticket, int32_t timeout_ms) {
    if (!S) return set_error(XM_EINVAL, "xm_serve_wait: NULL server");
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->tickets.find(ticket);
    if (it == S->tickets.end()) return set_error(XM_EINVAL, "xm_serve_wait: unknown ticket");
    Ticket* t = it->second;
    auto done = [&] { return t->state >= 2; };
    if (timeout_ms < 0) S->cv_done.wait(lk, done);
    else if (!S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), done))
        return set_error(XM_ETIMEOUT, "xm_serve_wait: ticket %lld still pending", (long long)ticket);
    if (t->state == 3) return set_error(t->status, "xm_serve_wait: ticket %lld failed", (long long)ticket);
    return XM_OK;
}

extern "C" xm_status xm_serve_result(xm_server* S, int64_t ticket, xm_batch_view* view) {
    if (!S || !view) return set_error(XM_EINVAL, "xm_serve_result: bad arguments");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->tickets.find(ticket);
    if (it == S->tickets.end()) return set_error(XM_EINVAL, "xm_serve_result: unknown ticket");
    Ticket* t = it->second;
    if (t->state != 2 || !t->hold || !t->hold->batch)
        return set_error(XM_EINVAL, "xm_serve_result: ticket %lld is not done", (long long)ticket);
    return xm_batch_get(t->hold->batch, t->index_in_batch, view);
}

extern "C" xm_status xm_serve_release(xm_server* S, int64_t ticket) {
    if (!S) return set_error(XM_EINVAL, "xm_serve_release: NULL server");
    xm_batch* to_free = nullptr;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        auto it = S->tickets.find(ticket);
        if (it == S->tickets.end()) return set_error(XM_EINVAL, "xm_serve_release: unknown ticket");
        Ticket* t = it->second;
        if (t->state < 2) return set_error(XM_EBUSY, "xm_serve_release: ticket %lld pending", (long long)ticket);
        if (t->hold && --t->hold->live == 0) {
            to_free = t->hold->batch;
            S->mem_in_use -= t->hold->est;
            t->hold->batch = nullptr;
        }
        S->tickets.erase(it);
        delete t;
    }
    if (to_free) xm_batch_free(to_free);
    S->cv_work.notify_all();
    return XM_OK;
}

extern "C" xm_status xm_serve_get_stats(xm_server* S, xm_serve_stats* out) {
    if (!S || !out) return set_error(XM_EINVAL, "xm_serve_get_stats: bad arguments");
    std::lock_guard<std::mutex> lk(S->mu);
    memset(out, 0, sizeof(*out));
    out->submitted = S->submitted;
    out->completed = S->completed;
    out->failed = S->failed;
    out->refused = S->refused;
    out->a_sources = S->a_sources;
    out->batches = S->batches;
    out->mem_in_use = S->mem_in_use;
    out->mem_budget = S->mem_budget;
    out->busy_s = S->busy_s + (S->active > 0
                                   ? std::chrono::duration<double>(Clock::now() - S->busy_since).count()
                                   : 0.0);
    if (!S->latency_ms.empty()) {
        std::vector<double> v = S->latency_ms;
        std::sort(v.begin(), v.end());
        auto q = [&](double f) {
            size_t k = (size_t)std::min<double>((double)v.size() - 1, f * (double)(v.size() - 1) + 0.5);
            return v[k];
        };
        out->p50_ms = q(0.50);
        out->p99_ms = q(0.99);
        out->max_ms = v.back();
    }
    return XM_OK;
}

extern "C" xm_status xm_serve_reset_stats(xm_server* S) {
    if (!S) return set_error(XM_EINVAL, "xm_serve_reset_stats: NULL server");
    std::lock_guard<std::mutex> lk(S->mu);
    const Clock::time_point now = Clock::now();
    S->window_start = now;
    S->submitted = S->completed = S->failed = S->refused = S->a_sources = S->batches = 0;
    S->latency_ms.clear();
    S->busy_s = 0.0;
    if (S->active > 0) S->busy_since = now;
    return XM_OK;
}

extern "C" xm_status xm_serve_close(xm_server* S) {
    if (!S) return XM_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stopping = true;
        for (Ticket* t : S->queue) {
            t->state = 3;
            t->status = XM_EBUSY;
        }
        S->queue.clear();
    }
    S->cv_work.notify_all();
    S->cv_done.notify_all();
    for (std::thread& w : S->workers) w.join();
    std::vector<xm_batch*> batches;
    for (auto& kv : S->tickets) {
        Ticket* t = kv.second;
        if (t->buf) dev_free(t->buf, S->copy_stream);
        if (t->hold && t->hold->batch) {
            batches.push_back(t->hold->batch);
            t->hold->batch = nullptr;
        }
        delete t;
    }
    S->tickets.clear();
    for (xm_batch* b : batches) xm_batch_free(b);
    for (cudaStream_t st : S->streams) {
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
    if (S->copy_stream) {
        cudaStreamSynchronize(S->copy_stream);
        cudaStreamDestroy(S->copy_stream);
    }
    delete S;
    return XM_OK;
}
