// ssp_server.cu -- the serving loop of include/ssp.h (ssp_server_*).
//
// Requests (one light curve each) are copied at submission into per-variant
// FIFO queues.  A launcher thread takes the queued requests of one variant,
// up to a points x frequencies cap, into one of two batch slots; it copies
// them into the slot's pinned buffer, then enqueues the H2D copy, the device
// pipeline of ssp_periodogram_device and the D2H copy of the powers and best
// periods on the slot's stream.  A completer thread waits for each slot in
// launch order and hands the results to the requests.  While one slot
// computes, the next batch is copied in, so the GPU is not left idle between
// batches.  Results are per (object, frequency) and do not depend on what
// else shares a batch.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "ssp_internal.h"

namespace {

using Clock = std::chrono::steady_clock;
using ssp_internal::fail;

constexpr double kDefaultBatchPtf = 4.0e9;
constexpr double kDefaultStallMs = 60000.0;
constexpr int64_t kDefaultInFlight = (int64_t)1 << 20;
constexpr int kSlots = 2;
constexpr int kVariants = 3;   // SSP_SS, SSP_SP, SSP_SPG

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

struct Request {
    int64_t ticket = 0;
    int variant = 0;
    std::vector<double> t, y, dy;
    Clock::time_point t_submit, t_done;
    int status = SSP_PENDING;   // guarded by the server mutex
    std::string err;
    std::vector<unsigned char> power;
    double best = 0.0;
};

// pinned host or device buffer that grows by doubling
struct Buf {
    unsigned char *p = nullptr;
    size_t cap = 0;
    bool host = false;
};

int buf_reserve(Buf &b, size_t bytes)
{
    if (bytes <= b.cap) return SSP_OK;
    const size_t cap = std::max(bytes, 2 * b.cap);
    if (b.p) {
        if (b.host) cudaFreeHost(b.p);
        else cudaFree(b.p);
        b.p = nullptr;
        b.cap = 0;
    }
    const cudaError_t e = b.host ? cudaHostAlloc((void **)&b.p, cap, cudaHostAllocDefault)
                                 : cudaMalloc((void **)&b.p, cap);
    if (e != cudaSuccess) {
        cudaGetLastError();
        b.p = nullptr;
        return fail(SSP_ERR_NOMEM, b.host ? "pinned batch buffer" : "device batch buffer");
    }
    b.cap = cap;
    return SSP_OK;
}

void buf_free(Buf &b)
{
    if (!b.p) return;
    if (b.host) cudaFreeHost(b.p);
    else cudaFree(b.p);
    b.p = nullptr;
    b.cap = 0;
}

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    Buf h_in, h_out, d_in, d_out;
    std::vector<std::shared_ptr<Request>> reqs;
    std::vector<int64_t> npo;
    size_t power_bytes = 0;    // offset of the best periods in h_out / d_out
    int status = SSP_OK;
    std::string err;
    bool busy = false;         // guarded by the server mutex
    Clock::time_point t_launch;   // when the batch's work was enqueued
};

}  // namespace

struct ssp_server {
    int device = 0;
    ssp_params P{};
    ssp_server_config cfg{};
    int64_t n_freq = 0;
    size_t rs = 4;             // bytes per power value
    double *d_freq = nullptr;

    std::mutex mu;
    std::condition_variable cv_launch, cv_complete, cv_done;
    std::deque<std::shared_ptr<Request>> queue[kVariants];
    double pending_ptf[kVariants] = {0.0, 0.0, 0.0};
    std::unordered_map<int64_t, std::shared_ptr<Request>> live;   // submitted, not collected
    std::deque<int64_t> finished;                                // not yet reported by next
    std::deque<int> launched;                                    // slots, in launch order
    Slot slots[kSlots];
    int64_t next_ticket = 1;
    bool stop = false;
    bool launcher_done = false;   // no batch will be launched any more
    std::thread launcher, completer;
};

namespace {

// fills slot sl with its batch and enqueues the work on the slot's stream
void launch_batch(ssp_server *S, Slot &sl, int variant)
{
    sl.t_launch = Clock::now();
    sl.status = SSP_OK;
    sl.err.clear();
    const int64_t nobj = (int64_t)sl.reqs.size();
    int64_t pts = 0;
    sl.npo.resize((size_t)nobj);
    for (int64_t i = 0; i < nobj; ++i) {
        sl.npo[(size_t)i] = (int64_t)sl.reqs[(size_t)i]->t.size();
        pts += sl.npo[(size_t)i];
    }
    const size_t in_col = align256(8 * (size_t)pts);
    sl.power_bytes = align256(S->rs * (size_t)nobj * (size_t)S->n_freq);
    const size_t out_bytes = sl.power_bytes + 8 * (size_t)nobj;
    int rc = buf_reserve(sl.h_in, 3 * in_col);
    if (!rc) rc = buf_reserve(sl.d_in, 3 * in_col);
    if (!rc) rc = buf_reserve(sl.h_out, out_bytes);
    if (!rc) rc = buf_reserve(sl.d_out, out_bytes);
    if (rc) {
        sl.status = rc;
        sl.err = ssp_internal::last_error();
        cudaEventRecord(sl.done, sl.stream);
        return;
    }
    double *ht = (double *)sl.h_in.p, *hy = (double *)(sl.h_in.p + in_col),
           *hdy = (double *)(sl.h_in.p + 2 * in_col);
    size_t at = 0;
    for (const auto &r : sl.reqs) {
        const size_t n = r->t.size();
        std::memcpy(ht + at, r->t.data(), 8 * n);
        std::memcpy(hy + at, r->y.data(), 8 * n);
        std::memcpy(hdy + at, r->dy.data(), 8 * n);
        at += n;
    }
    cudaError_t e = cudaMemcpyAsync(sl.d_in.p, sl.h_in.p, 3 * in_col, cudaMemcpyHostToDevice,
                                    sl.stream);
    if (e == cudaSuccess) {
        const double *dt = (const double *)sl.d_in.p;
        const double *dyv = (const double *)(sl.d_in.p + in_col);
        const double *ddy = (const double *)(sl.d_in.p + 2 * in_col);
        rc = ssp_internal::run(dt, dyv, ddy, sl.npo.data(), nobj, S->d_freq, S->n_freq,
                               (ssp_variant)variant, S->P, sl.d_out.p,
                               (double *)(sl.d_out.p + sl.power_bytes), sl.stream);
        if (rc) {
            sl.status = rc;
            sl.err = ssp_internal::last_error();
        } else {
            e = cudaMemcpyAsync(sl.h_out.p, sl.d_out.p, out_bytes, cudaMemcpyDeviceToHost,
                                sl.stream);
        }
    }
    if (e != cudaSuccess && sl.status == SSP_OK) {
        sl.status = SSP_ERR_CUDA;
        sl.err = std::string("batch copy: ") + cudaGetErrorString(e);
    }
    cudaEventRecord(sl.done, sl.stream);
}

int free_slot(const ssp_server *S)
{
    for (int k = 0; k < kSlots; ++k)
        if (!S->slots[k].busy) return k;
    return -1;
}

void launcher_loop(ssp_server *S, std::unique_lock<std::mutex> &lk)
{
    for (;;) {
        int slot = -1, v = -1;
        for (;;) {
            if (S->stop) return;
            slot = free_slot(S);
            // the variant whose oldest request has waited longest
            v = -1;
            for (int k = 0; k < kVariants; ++k)
                if (!S->queue[k].empty() &&
                    (v < 0 || S->queue[k].front()->t_submit < S->queue[v].front()->t_submit))
                    v = k;
            if (slot >= 0 && v >= 0) {
                const auto deadline = S->queue[v].front()->t_submit +
                                      std::chrono::duration_cast<Clock::duration>(
                                          std::chrono::duration<double, std::milli>(
                                              S->cfg.max_wait_ms));
                if (S->cfg.max_wait_ms > 0.0 && S->pending_ptf[v] < S->cfg.max_batch_ptf &&
                    Clock::now() < deadline) {
                    S->cv_launch.wait_until(lk, deadline);
                    continue;
                }
                break;
            }
            S->cv_launch.wait(lk);
        }
        Slot &sl = S->slots[slot];
        sl.reqs.clear();
        double ptf = 0.0;
        auto &q = S->queue[v];
        while (!q.empty()) {
            const double add = (double)q.front()->t.size() * (double)S->n_freq;
            if (!sl.reqs.empty() && ptf + add > S->cfg.max_batch_ptf) break;
            ptf += add;
            sl.reqs.push_back(q.front());
            q.pop_front();
        }
        S->pending_ptf[v] = q.empty() ? 0.0 : S->pending_ptf[v] - ptf;
        sl.busy = true;
        lk.unlock();
        launch_batch(S, sl, v);
        lk.lock();
        S->launched.push_back(slot);
        S->cv_complete.notify_one();
    }
}

void launcher_main(ssp_server *S)
{
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    launcher_loop(S, lk);
    S->launcher_done = true;
    S->cv_complete.notify_all();
}

void completer_main(ssp_server *S)
{
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        while (S->launched.empty() && !S->launcher_done) S->cv_complete.wait(lk);
        if (S->launched.empty()) return;   // the launcher has stopped and all is drained
        const int k = S->launched.front();
        S->launched.pop_front();
        Slot &sl = S->slots[k];
        lk.unlock();
        // Bounded wait for the batch: past stall_ms its requests end with
        // SSP_ERR_TIMEOUT at once, and the slot stays reserved until the GPU
        // has finished with its buffers.  (An injected stall takes the same
        // path after the batch completes normally.)
        const auto deadline = sl.t_launch + std::chrono::duration_cast<Clock::duration>(
                                                std::chrono::duration<double, std::milli>(
                                                    S->cfg.stall_ms));
        cudaError_t e = cudaEventQuery(sl.done);
        bool timed_out = false;
        while (e == cudaErrorNotReady) {
            if (Clock::now() >= deadline) {
                timed_out = true;
                break;
            }
            std::this_thread::sleep_for(std::chrono::microseconds(50));
            e = cudaEventQuery(sl.done);
        }
        if (ssp_internal::stall_injected()) timed_out = true;
        int status = sl.status;
        std::string err = sl.err;
        if (timed_out) {
            status = SSP_ERR_TIMEOUT;
            err = "batch did not finish within the server's stall limit";
        } else if (status == SSP_OK && e != cudaSuccess) {
            status = SSP_ERR_CUDA;
            err = std::string("batch: ") + cudaGetErrorString(e);
        }
        const auto now = Clock::now();
        const size_t row = S->rs * (size_t)S->n_freq;
        if (status == SSP_OK) {
            const double *best = (const double *)(sl.h_out.p + sl.power_bytes);
            for (size_t i = 0; i < sl.reqs.size(); ++i) {
                Request &r = *sl.reqs[i];
                r.power.assign(sl.h_out.p + i * row, sl.h_out.p + (i + 1) * row);
                r.best = best[i];
            }
        }
        lk.lock();
        for (const auto &r : sl.reqs) {
            r->status = status;
            r->err = err;
            r->t_done = now;
            r->t.clear();
            r->t.shrink_to_fit();
            r->y.clear();
            r->y.shrink_to_fit();
            r->dy.clear();
            r->dy.shrink_to_fit();
            if (S->live.count(r->ticket)) S->finished.push_back(r->ticket);
        }
        sl.reqs.clear();
        S->cv_done.notify_all();
        if (timed_out) {
            // the requests have their answer; the buffers are freed for the
            // next batch only once the GPU is done with them
            lk.unlock();
            cudaEventSynchronize(sl.done);
            lk.lock();
        }
        sl.busy = false;
        S->cv_launch.notify_one();
    }
}

void release(ssp_server *S)
{
    for (Slot &sl : S->slots) {
        buf_free(sl.h_in);
        buf_free(sl.h_out);
        buf_free(sl.d_in);
        buf_free(sl.d_out);
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.stream) cudaStreamDestroy(sl.stream);
    }
    if (S->d_freq) cudaFree(S->d_freq);
    delete S;
}

}  // namespace

extern "C" {

int ssp_server_create(const double *freq_grid, int64_t n_freq, const ssp_params *params,
                      const ssp_server_config *config, ssp_server **out)
{
    ssp_internal::clear_error();
    if (!out) return fail(SSP_ERR_ARG, "NULL server handle pointer");
    *out = nullptr;
    ssp_params P;
    ssp_default_params(&P);
    if (params) P = *params;
    int rc = ssp_internal::check_params(P);
    if (rc) return rc;
    rc = ssp_internal::check_freq(freq_grid, n_freq);
    if (rc) return rc;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(SSP_ERR_CUDA, "no CUDA device");
    }
    ssp_server *S = new ssp_server;
    S->device = dev;
    S->P = P;
    S->cfg.max_batch_ptf = kDefaultBatchPtf;
    S->cfg.max_wait_ms = 0.0;
    S->cfg.max_in_flight = kDefaultInFlight;
    S->cfg.stall_ms = kDefaultStallMs;
    if (config) {
        if (config->stall_ms > 0.0) S->cfg.stall_ms = config->stall_ms;
        if (config->max_batch_ptf > 0.0) S->cfg.max_batch_ptf = config->max_batch_ptf;
        if (config->max_wait_ms > 0.0) S->cfg.max_wait_ms = config->max_wait_ms;
        if (config->max_in_flight > 0) S->cfg.max_in_flight = config->max_in_flight;
    }
    S->n_freq = n_freq;
    S->rs = P.precision == SSP_FP64 ? 8 : 4;
    e = cudaMalloc((void **)&S->d_freq, 8 * (size_t)n_freq);
    if (e == cudaSuccess)
        e = cudaMemcpy(S->d_freq, freq_grid, 8 * (size_t)n_freq, cudaMemcpyHostToDevice);
    for (int k = 0; k < kSlots && e == cudaSuccess; ++k) {
        Slot &sl = S->slots[k];
        sl.h_in.host = sl.h_out.host = true;
        e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        release(S);
        return fail(SSP_ERR_CUDA, cudaGetErrorString(e));
    }
    S->launcher = std::thread(launcher_main, S);
    S->completer = std::thread(completer_main, S);
    *out = S;
    return SSP_OK;
}

int ssp_server_submit(ssp_server *s, const double *t, const double *y, const double *dy,
                      int64_t n, ssp_variant variant, int64_t *out_ticket)
{
    ssp_internal::clear_error();
    if (!s || !out_ticket) return fail(SSP_ERR_ARG, "NULL server or ticket pointer");
    if (variant != SSP_SS && variant != SSP_SP && variant != SSP_SPG)
        return fail(SSP_ERR_ARG, "unknown variant");
    int rc = ssp_internal::check_one_object(s->P, t, y, dy, n);
    if (rc) return rc;
    auto r = std::make_shared<Request>();
    r->variant = (int)variant;
    r->t.assign(t, t + n);
    r->y.assign(y, y + n);
    r->dy.assign(dy, dy + n);
    std::lock_guard<std::mutex> lk(s->mu);
    if ((int64_t)s->live.size() >= s->cfg.max_in_flight)
        return fail(SSP_ERR_BUSY, "max_in_flight requests are submitted and not yet collected");
    r->ticket = s->next_ticket++;
    r->t_submit = Clock::now();
    s->live[r->ticket] = r;
    s->queue[r->variant].push_back(r);
    s->pending_ptf[r->variant] += (double)n * (double)s->n_freq;
    *out_ticket = r->ticket;
    s->cv_launch.notify_one();
    return SSP_OK;
}

int ssp_server_next(ssp_server *s, int wait_ms, int64_t *out_ticket)
{
    ssp_internal::clear_error();
    if (!s || !out_ticket) return fail(SSP_ERR_ARG, "NULL server or ticket pointer");
    std::unique_lock<std::mutex> lk(s->mu);
    const auto deadline = Clock::now() + std::chrono::milliseconds(std::max(0, wait_ms));
    for (;;) {
        while (!s->finished.empty() && !s->live.count(s->finished.front())) s->finished.pop_front();
        if (!s->finished.empty()) {
            *out_ticket = s->finished.front();
            s->finished.pop_front();
            return SSP_OK;
        }
        if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout) {
            while (!s->finished.empty() && !s->live.count(s->finished.front()))
                s->finished.pop_front();
            if (s->finished.empty()) return SSP_PENDING;
        }
    }
}

int ssp_server_poll(ssp_server *s, int64_t ticket, int wait_ms, void *out_power,
                    double *out_best_period, double *out_latency_ms)
{
    ssp_internal::clear_error();
    if (!s) return fail(SSP_ERR_ARG, "NULL server");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->live.find(ticket);
    if (it == s->live.end()) return fail(SSP_ERR_ARG, "unknown or retired ticket");
    std::shared_ptr<Request> r = it->second;
    s->cv_done.wait_for(lk, std::chrono::milliseconds(std::max(0, wait_ms)),
                        [&] { return r->status != SSP_PENDING; });
    if (r->status == SSP_PENDING) return SSP_PENDING;
    s->live.erase(ticket);
    if (r->status != SSP_OK) return fail(r->status, r->err.c_str());
    if (out_power) std::memcpy(out_power, r->power.data(), r->power.size());
    if (out_best_period) *out_best_period = r->best;
    if (out_latency_ms)
        *out_latency_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
    return SSP_OK;
}

int ssp_server_destroy(ssp_server *s)
{
    ssp_internal::clear_error();
    if (!s) return fail(SSP_ERR_ARG, "NULL server");
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        for (auto &q : s->queue) q.clear();
        s->cv_launch.notify_all();
        s->cv_complete.notify_all();
        s->cv_done.notify_all();
    }
    if (s->launcher.joinable()) s->launcher.join();
    if (s->completer.joinable()) s->completer.join();
    release(s);
    return SSP_OK;
}

}  // extern "C"
