// ssp_server.cu -- the serving loop of include/ssp.h (ssp_server_*): continuous
// batching of single light curves under a device-memory budget.
//
// Admission.  A submitted request waits in a host queue until its inputs fit
// the device arena of its variant: one ring buffer per variant in device
// memory (t, y, dy as three arrays), sized from the server's byte budget.
// Admitted requests are uploaded into the ring at once (upload stream) and
// stay resident there until their batch has finished, so a batch reads its
// inputs in place: consecutive admitted requests of one variant are
// contiguous in the ring, which is the CSR layout the device pipeline takes.
//
// Batching.  A worker forms a batch from the oldest admitted requests of one
// variant (up to max_batch_ptf points x frequencies, never across the ring's
// wrap) whenever one of `slots` batch slots is free, and launches the device
// pipeline of ssp_periodogram_device on the slot's stream after the uploads
// it reads.  Several slots run at once, so requests that arrive while other
// batches are on the GPU start as soon as a slot and memory allow, and their
// kernels overlap.
//
// Completion.  A second worker watches every slot's completion event and
// hands each finished batch's results to its requests in completion order
// (a short batch that started after a long one may finish first).  A batch
// still running stall_ms after its launch ends its requests with
// SSP_ERR_TIMEOUT; its slot and ring space are released only once the GPU
// has finished with them.  Results are per (object, frequency) and do not
// depend on what else shares a batch.
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
constexpr int64_t kDefaultInFlight = (int64_t)1 << 20;
constexpr double kDefaultStallMs = 60000.0;
constexpr int kDefaultSlots = 4;
constexpr int kMaxSlots = 16;
constexpr double kDefaultArenaBytes = 768.0 * 1024 * 1024;   // all variants together
constexpr int kVariants = 3;   // SSP_SS, SSP_SP, SSP_SPG

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

struct Request {
    int64_t ticket = 0;
    int variant = 0;
    int64_t n = 0;
    std::vector<double> t, y, dy;   // host copy until uploaded
    int64_t pos = -1;               // position in its ring (virtual, increasing), once admitted
    bool launched = false;          // in a batch on the GPU (or finished)
    bool released = false;          // its batch finished: ring space reusable
    Clock::time_point t_submit, t_done;
    int status = SSP_PENDING;       // guarded by the server mutex
    std::string err;
    std::vector<unsigned char> power;
    double best = 0.0;
};

// Ring of points in device memory for one variant.  Positions are virtual
// (they only grow); a request occupies [pos, pos + n), physically
// pos % cap .. (pos % cap) + n, never across the end of the buffer.
struct Ring {
    double *t = nullptr, *y = nullptr, *dy = nullptr;
    int64_t cap = 0;                 // points
    int64_t head = 0, tail = 0;      // next free position; start of live data
    std::deque<std::shared_ptr<Request>> live;   // admitted, in ring order
    // where a request of n points would go, or -1 if the ring lacks room now
    int64_t place(int64_t n) const
    {
        int64_t p = head;
        if (p % cap + n > cap) p += cap - p % cap;   // skip the end of the buffer
        return (p + n - tail <= cap) ? p : -1;
    }
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
    cudaEvent_t uploaded = nullptr;   // recorded on the upload stream at launch
    cudaEvent_t done = nullptr;
    Buf h_out, d_out;
    std::vector<std::shared_ptr<Request>> reqs;
    std::vector<int64_t> npo;
    int variant = 0;
    size_t power_bytes = 0;    // offset of the best periods in h_out / d_out
    int status = SSP_OK;
    std::string err;
    bool busy = false;         // guarded by the server mutex
    bool enqueued = false;     // launch_batch has returned: `done` marks this batch
    bool answered = false;     // its requests have their status (a timeout answers early)
    Clock::time_point t_launch;
};

}  // namespace

struct ssp_server {
    int device = 0;
    ssp_params P{};
    ssp_server_config cfg{};
    int64_t n_freq = 0;
    size_t rs = 4;             // bytes per power value
    double *d_freq = nullptr;
    int nslots = kDefaultSlots;
    cudaStream_t upload = nullptr;

    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<Request>> waiting[kVariants];   // submitted, not yet admitted
    Ring ring[kVariants];
    std::unordered_map<int64_t, std::shared_ptr<Request>> live;   // submitted, not collected
    std::deque<int64_t> finished;                                // not yet reported by next
    Slot slots[kMaxSlots];
    int in_flight = 0;         // busy slots
    int64_t next_ticket = 1;
    bool stop = false;
    bool launcher_done = false;   // no batch will be launched any more
    std::thread launcher, completer;
};

namespace {

// Drops the finished requests at the start of a ring's live list: their
// space is free.
void pop_released(Ring &rg)
{
    while (!rg.live.empty() && rg.live.front()->released) {
        rg.live.pop_front();
        rg.tail = rg.live.empty() ? rg.head : rg.live.front()->pos;
    }
}

// Admits waiting requests, oldest first across variants, while their ring has
// room; uploads each into its ring.  Called by the launcher with the lock
// held; releases it around the copies.
void admit(ssp_server *S, std::unique_lock<std::mutex> &lk)
{
    for (;;) {
        int v = -1;
        for (int k = 0; k < kVariants; ++k)
            if (!S->waiting[k].empty() &&
                (v < 0 || S->waiting[k].front()->t_submit < S->waiting[v].front()->t_submit))
                v = k;
        if (v < 0) return;
        Ring &rg = S->ring[v];
        const auto r = S->waiting[v].front();
        const int64_t p = rg.place(r->n);
        if (p < 0) return;   // the oldest waits for room: admission stays in order
        S->waiting[v].pop_front();
        r->pos = p;
        rg.head = p + r->n;
        rg.live.push_back(r);
        lk.unlock();
        const size_t at = (size_t)(p % rg.cap), bytes = 8 * (size_t)r->n;
        cudaError_t e = ssp_internal::upload_fault_injected()
                            ? cudaErrorInvalidValue
                            : cudaMemcpyAsync(rg.t + at, r->t.data(), bytes, cudaMemcpyHostToDevice,
                                              S->upload);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(rg.y + at, r->y.data(), bytes, cudaMemcpyHostToDevice, S->upload);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(rg.dy + at, r->dy.data(), bytes, cudaMemcpyHostToDevice, S->upload);
        // (copies from pageable memory are staged before the calls return)
        std::vector<double>().swap(r->t);
        std::vector<double>().swap(r->y);
        std::vector<double>().swap(r->dy);
        lk.lock();
        if (e != cudaSuccess) {
            // answered at once and never batched (batches stop at it); its
            // ring space is reused once the requests before it are done
            cudaGetLastError();
            r->status = SSP_ERR_CUDA;
            r->err = std::string("upload: ") + cudaGetErrorString(e);
            r->launched = r->released = true;
            r->t_done = Clock::now();
            if (S->live.count(r->ticket)) S->finished.push_back(r->ticket);
            pop_released(rg);
            S->cv_done.notify_all();
        }
    }
}

// oldest admitted, not yet launched request of variant v, as an index into
// its ring's live list, or -1
int64_t first_unlaunched(const Ring &rg)
{
    for (size_t i = 0; i < rg.live.size(); ++i)
        if (!rg.live[i]->launched) return (int64_t)i;
    return -1;
}

int free_slot(const ssp_server *S)
{
    for (int k = 0; k < S->nslots; ++k)
        if (!S->slots[k].busy) return k;
    return -1;
}

// Enqueues slot sl's batch (its requests lie contiguously in the ring of its
// variant) on the slot's stream, after the uploads it reads.
void launch_batch(ssp_server *S, Slot &sl)
{
    sl.t_launch = Clock::now();
    sl.status = SSP_OK;
    sl.err.clear();
    Ring &rg = S->ring[sl.variant];
    const int64_t nobj = (int64_t)sl.reqs.size();
    sl.npo.resize((size_t)nobj);
    for (int64_t i = 0; i < nobj; ++i) sl.npo[(size_t)i] = sl.reqs[(size_t)i]->n;
    sl.power_bytes = align256(S->rs * (size_t)nobj * (size_t)S->n_freq);
    const size_t out_bytes = sl.power_bytes + 8 * (size_t)nobj;
    int rc = buf_reserve(sl.h_out, out_bytes);
    if (!rc) rc = buf_reserve(sl.d_out, out_bytes);
    cudaError_t e = cudaSuccess;
    if (!rc) {
        e = cudaEventRecord(sl.uploaded, S->upload);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(sl.stream, sl.uploaded, 0);
    }
    if (!rc && e == cudaSuccess) {
        const size_t at = (size_t)(sl.reqs.front()->pos % rg.cap);
        rc = ssp_internal::run(rg.t + at, rg.y + at, rg.dy + at, sl.npo.data(), nobj, S->d_freq,
                               S->n_freq, (ssp_variant)sl.variant, S->P, sl.d_out.p,
                               (double *)(sl.d_out.p + sl.power_bytes), sl.stream);
        if (!rc)
            e = cudaMemcpyAsync(sl.h_out.p, sl.d_out.p, out_bytes, cudaMemcpyDeviceToHost, sl.stream);
    }
    if (rc) {
        sl.status = rc;
        sl.err = ssp_internal::last_error();
    } else if (e != cudaSuccess) {
        cudaGetLastError();
        sl.status = SSP_ERR_CUDA;
        sl.err = std::string("batch: ") + cudaGetErrorString(e);
    }
    cudaEventRecord(sl.done, sl.stream);
}

void launcher_loop(ssp_server *S, std::unique_lock<std::mutex> &lk)
{
    for (;;) {
        int slot = -1, v = -1;
        int64_t first = -1;
        for (;;) {
            if (S->stop) return;
            admit(S, lk);
            if (S->stop) return;
            slot = free_slot(S);
            // the variant whose oldest admitted request has waited longest
            v = -1;
            first = -1;
            for (int k = 0; k < kVariants; ++k) {
                const int64_t f = first_unlaunched(S->ring[k]);
                if (f >= 0 && (v < 0 || S->ring[k].live[(size_t)f]->t_submit <
                                            S->ring[v].live[(size_t)first]->t_submit)) {
                    v = k;
                    first = f;
                }
            }
            if (slot >= 0 && v >= 0) {
                const auto r0 = S->ring[v].live[(size_t)first];
                const auto deadline = r0->t_submit + std::chrono::duration_cast<Clock::duration>(
                                                         std::chrono::duration<double, std::milli>(
                                                             S->cfg.max_wait_ms));
                double ptf = 0.0;
                for (size_t i = (size_t)first; i < S->ring[v].live.size(); ++i)
                    ptf += (double)S->ring[v].live[i]->n * (double)S->n_freq;
                if (S->cfg.max_wait_ms > 0.0 && ptf < S->cfg.max_batch_ptf && Clock::now() < deadline) {
                    S->cv_work.wait_until(lk, deadline);
                    continue;
                }
                break;
            }
            S->cv_work.wait(lk);
        }
        Slot &sl = S->slots[slot];
        Ring &rg = S->ring[v];
        sl.reqs.clear();
        sl.variant = v;
        double ptf = 0.0;
        int64_t end = -1;
        for (size_t i = (size_t)first; i < rg.live.size(); ++i) {
            const auto &r = rg.live[i];
            // not yet launched (a failed upload is answered and never
            // batched), contiguous in the ring, and within the cap (at least
            // one request)
            if (r->launched || (end >= 0 && r->pos != end)) break;
            const double add = (double)r->n * (double)S->n_freq;
            if (!sl.reqs.empty() && ptf + add > S->cfg.max_batch_ptf) break;
            ptf += add;
            end = r->pos + r->n;
            r->launched = true;
            sl.reqs.push_back(r);
        }
        sl.busy = true;
        sl.enqueued = false;
        sl.answered = false;
        ++S->in_flight;
        lk.unlock();
        launch_batch(S, sl);
        lk.lock();
        sl.enqueued = true;
        S->cv_done.notify_all();   // wakes the completer
    }
}

void launcher_main(ssp_server *S)
{
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    launcher_loop(S, lk);
    S->launcher_done = true;
    S->cv_done.notify_all();
}

// Hands slot sl's outcome to its requests (status, and results when OK).
// Lock held.
void answer(ssp_server *S, Slot &sl, int status, const std::string &err)
{
    const auto now = Clock::now();
    const size_t row = S->rs * (size_t)S->n_freq;
    const double *best = (const double *)(sl.h_out.p + sl.power_bytes);
    for (size_t i = 0; i < sl.reqs.size(); ++i) {
        Request &r = *sl.reqs[i];
        if (status == SSP_OK) {
            r.power.assign(sl.h_out.p + i * row, sl.h_out.p + (i + 1) * row);
            r.best = best[i];
        }
        r.status = status;
        r.err = err;
        r.t_done = now;
        if (S->live.count(r.ticket)) S->finished.push_back(r.ticket);
    }
    sl.answered = true;
    S->cv_done.notify_all();
}

// The GPU has finished with slot sl: its ring space and the slot are free.
// Lock held.
void release_slot(ssp_server *S, Slot &sl)
{
    for (const auto &r : sl.reqs) r->released = true;
    pop_released(S->ring[sl.variant]);
    sl.reqs.clear();
    sl.busy = false;
    sl.enqueued = false;
    --S->in_flight;
    S->cv_work.notify_all();   // a slot and ring space for the launcher
}

void completer_main(ssp_server *S)
{
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        while (S->in_flight == 0 && !S->launcher_done) S->cv_done.wait(lk);
        if (S->in_flight == 0) return;   // the launcher has stopped and all is drained
        bool progress = false;
        for (int k = 0; k < S->nslots; ++k) {
            Slot &sl = S->slots[k];
            if (!sl.busy || !sl.enqueued) continue;   // (a batch still being enqueued)
            lk.unlock();
            const cudaError_t e = cudaEventQuery(sl.done);
            lk.lock();
            if (e == cudaErrorNotReady) {
                // bounded wait: past stall_ms the requests are answered now,
                // the slot is freed when the GPU is done with it
                if (!sl.answered &&
                    Clock::now() >= sl.t_launch + std::chrono::duration_cast<Clock::duration>(
                                                      std::chrono::duration<double, std::milli>(
                                                          S->cfg.stall_ms))) {
                    answer(S, sl, SSP_ERR_TIMEOUT,
                           "batch did not finish within the server's stall limit");
                    progress = true;
                }
                continue;
            }
            if (!sl.answered) {
                int status = sl.status;
                std::string err = sl.err;
                if (ssp_internal::stall_injected()) {
                    status = SSP_ERR_TIMEOUT;
                    err = "batch did not finish within the server's stall limit";
                } else if (status == SSP_OK && e != cudaSuccess) {
                    cudaGetLastError();
                    status = SSP_ERR_CUDA;
                    err = std::string("batch: ") + cudaGetErrorString(e);
                }
                answer(S, sl, status, err);
            }
            release_slot(S, sl);
            progress = true;
        }
        if (!progress) {
            lk.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(50));
            lk.lock();
        }
    }
}

void release(ssp_server *S)
{
    for (int k = 0; k < kMaxSlots; ++k) {
        Slot &sl = S->slots[k];
        buf_free(sl.h_out);
        buf_free(sl.d_out);
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.uploaded) cudaEventDestroy(sl.uploaded);
        if (sl.stream) cudaStreamDestroy(sl.stream);
    }
    for (Ring &rg : S->ring)
        if (rg.t) cudaFree(rg.t);
    if (S->upload) cudaStreamDestroy(S->upload);
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
    if (config && config->slots > kMaxSlots)
        return fail(SSP_ERR_ARG, "at most 16 batch slots");
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
    S->cfg.slots = kDefaultSlots;
    S->cfg.device_bytes = kDefaultArenaBytes;
    if (config) {
        if (config->max_batch_ptf > 0.0) S->cfg.max_batch_ptf = config->max_batch_ptf;
        if (config->max_wait_ms > 0.0) S->cfg.max_wait_ms = config->max_wait_ms;
        if (config->max_in_flight > 0) S->cfg.max_in_flight = config->max_in_flight;
        if (config->stall_ms > 0.0) S->cfg.stall_ms = config->stall_ms;
        if (config->slots > 0) S->cfg.slots = config->slots;
        if (config->device_bytes > 0.0) S->cfg.device_bytes = config->device_bytes;
    }
    S->nslots = (int)S->cfg.slots;
    S->n_freq = n_freq;
    S->rs = P.precision == SSP_FP64 ? 8 : 4;
    e = cudaMalloc((void **)&S->d_freq, 8 * (size_t)n_freq);
    if (e == cudaSuccess)
        e = cudaMemcpy(S->d_freq, freq_grid, 8 * (size_t)n_freq, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->upload, cudaStreamNonBlocking);
    // the arena: one ring per variant, t, y and dy of 8 bytes a point each
    const int64_t cap = std::max<int64_t>(4, (int64_t)(S->cfg.device_bytes / (kVariants * 24.0)));
    for (int v = 0; v < kVariants && e == cudaSuccess; ++v) {
        Ring &rg = S->ring[v];
        rg.cap = cap;
        e = cudaMalloc((void **)&rg.t, 24 * (size_t)cap);
        if (e == cudaSuccess) {
            rg.y = rg.t + cap;
            rg.dy = rg.t + 2 * cap;
        }
    }
    for (int k = 0; k < S->nslots && e == cudaSuccess; ++k) {
        Slot &sl = S->slots[k];
        sl.h_out.host = true;
        e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.uploaded, cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        const int code = e == cudaErrorMemoryAllocation ? SSP_ERR_NOMEM : SSP_ERR_CUDA;
        cudaGetLastError();
        release(S);
        return fail(code, cudaGetErrorString(e));
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
    if (n > s->ring[variant].cap)
        return fail(SSP_ERR_NOMEM, "object larger than the server's device arena for its variant");
    auto r = std::make_shared<Request>();
    r->variant = (int)variant;
    r->n = n;
    r->t.assign(t, t + n);
    r->y.assign(y, y + n);
    r->dy.assign(dy, dy + n);
    std::lock_guard<std::mutex> lk(s->mu);
    if ((int64_t)s->live.size() >= s->cfg.max_in_flight)
        return fail(SSP_ERR_BUSY, "max_in_flight requests are submitted and not yet collected");
    r->ticket = s->next_ticket++;
    r->t_submit = Clock::now();
    s->live[r->ticket] = r;
    s->waiting[r->variant].push_back(r);
    *out_ticket = r->ticket;
    s->cv_work.notify_all();
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
        for (auto &q : s->waiting) q.clear();
        s->cv_work.notify_all();
        s->cv_done.notify_all();
    }
    // the launcher stops; the completer drains the batches already on the GPU
    if (s->launcher.joinable()) s->launcher.join();
    if (s->completer.joinable()) s->completer.join();
    release(s);
    return SSP_OK;
}

}  // extern "C"
