// sg_serve.cpp -- request loop with continuous batching on one GPU.
//
// Requests (L, h, temperature ladder, coupling distribution, sample count,
// seed, sweeps) arrive at any time from any host thread. One worker thread
// owns the device work: it admits queued requests while their ensembles fit
// the device-memory budget, keeps every admitted ensemble (lattices, couplings,
// accumulators, sweep counters) resident on the device, and advances each on
// its own stream in chunks of sweeps, so the kernels of all resident requests
// share the GPU. A request that arrives while others run starts at once if
// memory allows; a finished one leaves as soon as its last chunk completes,
// its accumulators are copied out and its memory is released for the queue.
// Results do not depend on the mix: each ensemble's chain is keyed by its own
// seed and sweep index.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "sg_internal.h"

namespace {

double now_s()
{
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

enum { RQ_QUEUED = 0, RQ_RUNNING = 1, RQ_DONE = 2, RQ_FAILED = 3, RQ_CANCELLED = 4 };

// A chunk is at most this many spin-flip attempts (~10 ms of GPU time), so a
// large request never holds the SMs long enough to stall the small ones.
constexpr double kChunkAttempts = 2.0e9;

struct Request {
    sg_request r{};
    std::vector<double> T;
    int state = RQ_QUEUED;
    sg_status err = SG_OK;
    std::string err_msg;
    sg_ensemble *e = nullptr;
    cudaStream_t st = nullptr;  // the request's own stream
    cudaEvent_t ev = nullptr;   // completion of its chunk in flight
    bool inflight = false;
    int64_t chunk = 0;
    double chunk_attempts = 0;
    size_t bytes = 0;
    int64_t remaining = 0;
    bool cancel = false;
    std::vector<double> acc;
    double t_submit = 0, t_start = 0, t_done = 0;
};

}  // namespace

struct sg_server {
    sg_server_options opt{};
    cudaStream_t stream = nullptr;
    int device = 0;
    std::thread worker;
    std::mutex mu;
    std::condition_variable cv;       // wakes the worker
    std::condition_variable done_cv;  // wakes waiters
    std::deque<int64_t> queue;
    std::map<int64_t, Request> reqs;
    std::vector<int64_t> active;
    bool stop = false;  // set by destroy
    size_t used = 0;
    int64_t next_id = 1;
    // statistics
    int64_t completed = 0, rounds = 0;
    double attempts = 0, busy_s = 0;
    double busy_since = -1.0;  // start of the current busy interval, or -1
    std::vector<double> latencies;
};

namespace {

sg_options request_options(const sg_request &r)
{
    sg_options o;
    sg_options_default(&o);
    const bool msc_ok = r.dist == (int32_t)SG_PM_J && r.n_samples % 64 == 0 && r.L <= 16;
    o.layout = (r.layout == SG_LAYOUT_INT8 || r.layout == SG_LAYOUT_MSC64)
                   ? r.layout
                   : (msc_ok ? SG_LAYOUT_MSC64 : SG_LAYOUT_INT8);
    o.n_therm = r.n_therm >= 0 ? r.n_therm : r.n_sweeps / 2;  // thermalise for the first half
    o.exchange_every = r.exchange_every > 0 ? r.exchange_every : 1;
    o.measure_every = r.measure_every > 0 ? r.measure_every : 1;
    return o;
}

// Release a request's device resources (called without the lock).
void release_request(Request &q)
{
    if (q.e) sg_destroy(q.e);
    if (q.ev) cudaEventDestroy(q.ev);
    if (q.st) cudaStreamDestroy(q.st);
    q.e = nullptr;
    q.ev = nullptr;
    q.st = nullptr;
}

// Worker: admission, then every resident request advances on its own stream
// chunk by chunk; finished chunks are found by polling their events, so a
// short request leaves as soon as its own work is done and a new one starts
// at once (continuous batching).
void worker_loop(sg_server *sv)
{
    cudaSetDevice(sv->device);
    std::unique_lock<std::mutex> lk(sv->mu);
    double &busy_since = sv->busy_since;
    for (;;) {
        // ---- admission: queued requests while their ensembles fit the budget
        while (!sv->queue.empty() && !sv->stop) {
            const int64_t id = sv->queue.front();
            Request &q = sv->reqs[id];
            if (q.cancel) {
                sv->queue.pop_front();
                q.state = RQ_CANCELLED;
                q.t_done = now_s();
                sv->done_cv.notify_all();
                continue;
            }
            if (sv->opt.max_active > 0 && (int)sv->active.size() >= sv->opt.max_active) break;
            const sg_options o = request_options(q.r);
            const size_t need =
                sg_ensemble_bytes(q.r.L, q.r.n_T, q.r.n_samples, (sg_coupling)q.r.dist, &o);
            if (need == 0 || (sv->used + need > sv->opt.memory_budget && sv->active.empty())) {
                sv->queue.pop_front();
                q.state = RQ_FAILED;
                q.err = need == 0 ? SG_EINVAL : SG_ENOMEM;
                q.err_msg = need == 0 ? "request rejected by sg_ensemble_bytes"
                                      : "request larger than the server's memory budget";
                q.t_done = now_s();
                sv->done_cv.notify_all();
                continue;
            }
            if (sv->used + need > sv->opt.memory_budget) break;  // wait for memory, in order
            sv->queue.pop_front();
            const sg_request r = q.r;
            const std::vector<double> T = q.T;
            lk.unlock();
            cudaStream_t st = nullptr;
            cudaEvent_t ev = nullptr;
            sg_ensemble *e = nullptr;
            sg_status rc = SG_OK;
            // smaller requests get higher-priority streams: when SMs free up,
            // the scheduler prefers their CTAs (shortest work first)
            int least = 0, greatest = 0;
            cudaDeviceGetStreamPriorityRange(&least, &greatest);
            const double work = (double)r.L * r.L * r.L * 2.0 * r.n_T * (double)r.n_samples *
                                (double)std::max<int64_t>(r.n_sweeps, 1);
            int bucket = (int)std::floor(std::log10(std::max(work, 1.0))) - 9;
            bucket = std::max(0, bucket);
            const int prio = std::min(least, greatest + bucket);
            if (cudaStreamCreateWithPriority(&st, cudaStreamNonBlocking, prio) != cudaSuccess ||
                cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess)
                rc = SG_ECUDA;
            if (rc == SG_OK)
                rc = sg_create_ensemble(r.L, r.h, T.data(), r.n_T, (sg_coupling)r.dist,
                                        r.n_samples, r.seed, &o, nullptr, nullptr, st, &e);
            const std::string msg = rc == SG_OK ? "" : sg_last_error();
            lk.lock();
            Request &q2 = sv->reqs[id];
            q2.st = st;
            q2.ev = ev;
            if (rc != SG_OK) {
                lk.unlock();
                release_request(q2);
                lk.lock();
                if (rc == SG_ENOMEM && !sv->active.empty()) {
                    sv->queue.push_front(id);  // retry once memory frees up
                    break;
                }
                q2.state = RQ_FAILED;
                q2.err = rc;
                q2.err_msg = msg;
                q2.t_done = now_s();
                sv->done_cv.notify_all();
                continue;
            }
            q2.e = e;
            q2.bytes = need;
            q2.remaining = r.n_sweeps;
            q2.state = RQ_RUNNING;
            q2.t_start = now_s();
            sv->used += need;
            sv->active.push_back(id);
        }
        if (sv->stop) break;
        if (sv->active.empty()) {
            if (busy_since >= 0) {
                sv->busy_s += now_s() - busy_since;
                busy_since = -1.0;
            }
            sv->cv.wait(lk, [&] { return sv->stop || !sv->queue.empty(); });
            if (sv->stop) break;
            continue;
        }
        if (busy_since < 0) busy_since = now_s();
        // ---- launch the next chunk of every idle request
        const int64_t chunk = sv->opt.chunk_sweeps > 0 ? sv->opt.chunk_sweeps : 256;
        for (int64_t id : sv->active) {
            Request &q = sv->reqs[id];
            if (q.inflight || q.cancel || q.remaining <= 0) continue;
            sg_info inf;
            sg_get_info(q.e, &inf);
            const int64_t cap = std::max<int64_t>(
                1, (int64_t)(kChunkAttempts / (double)std::max<int64_t>(inf.attempts_per_sweep, 1)));
            const int64_t n = std::min(std::min(chunk, cap), q.remaining);
            sg_ensemble *e = q.e;
            lk.unlock();
            sg_status rc = sv->opt.use_graph ? sg_sweep_batch(&e, 1, n, 1) : sg_sweep(e, n);
            cudaError_t ce = rc == SG_OK ? cudaEventRecord(q.ev, q.st) : cudaSuccess;
            lk.lock();
            if (rc != SG_OK || ce != cudaSuccess) {
                q.state = RQ_FAILED;
                q.err = rc != SG_OK ? rc : SG_ECUDA;
                q.err_msg = rc != SG_OK ? sg_last_error() : cudaGetErrorString(ce);
                q.cancel = true;  // retired below
                continue;
            }
            q.inflight = true;
            q.chunk = n;
            q.chunk_attempts = (double)inf.attempts_per_sweep * (double)n;
            sv->rounds += 1;
        }
        // ---- retire finished, failed and cancelled requests
        bool progressed = false;
        std::vector<int64_t> keep;
        for (int64_t id : sv->active) {
            Request &q = sv->reqs[id];
            if (q.inflight) {
                const cudaError_t qe = cudaEventQuery(q.ev);
                if (qe == cudaErrorNotReady) {
                    keep.push_back(id);
                    continue;
                }
                q.inflight = false;
                progressed = true;
                if (qe != cudaSuccess) {
                    q.state = RQ_FAILED;
                    q.err = SG_ECUDA;
                    q.err_msg = cudaGetErrorString(qe);
                    q.cancel = true;
                } else {
                    q.remaining -= q.chunk;
                    sv->attempts += q.chunk_attempts;
                }
            }
            bool finish = false;
            if (q.state == RQ_FAILED) {
                finish = true;
            } else if (q.cancel) {
                q.state = RQ_CANCELLED;
                finish = true;
            } else if (q.remaining <= 0) {
                sg_info inf;
                sg_get_info(q.e, &inf);
                q.acc.assign((size_t)inf.n_samples * inf.n_T * SG_NACC, 0.0);
                sg_ensemble *e = q.e;
                lk.unlock();
                const sg_status gs = sg_get_accumulators(e, q.acc.data());
                lk.lock();
                q.state = gs == SG_OK ? RQ_DONE : RQ_FAILED;
                q.err = gs;
                finish = true;
            }
            if (finish) {
                q.t_done = now_s();
                if (q.state == RQ_DONE) {
                    sv->completed += 1;
                    sv->latencies.push_back(q.t_done - q.t_submit);
                }
                sv->used -= q.bytes;
                q.bytes = 0;
                lk.unlock();
                release_request(q);
                lk.lock();
                sv->done_cv.notify_all();
                progressed = true;
            } else {
                keep.push_back(id);
            }
        }
        sv->active = keep;
        if (!progressed) {  // nothing finished: give the GPU a moment
            lk.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(100));
            lk.lock();
        }
    }
    // shutdown: wait for in-flight work and release what is still resident
    for (int64_t id : sv->active) {
        Request &q = sv->reqs[id];
        if (q.st) cudaStreamSynchronize(q.st);
        release_request(q);
        q.state = RQ_CANCELLED;
    }
    sv->active.clear();
    sv->done_cv.notify_all();
}

double percentile(std::vector<double> v, double p)
{
    if (v.empty()) return NAN;
    std::sort(v.begin(), v.end());
    const double pos = p * (double)(v.size() - 1);
    const size_t lo = (size_t)pos;
    const size_t hi = std::min(lo + 1, v.size() - 1);
    return v[lo] + (pos - (double)lo) * (v[hi] - v[lo]);
}

}  // namespace

extern "C" {

void sg_server_options_default(sg_server_options *o)
{
    if (!o) return;
    *o = sg_server_options{};
    o->memory_budget = 0;
    o->max_active = 0;
    o->chunk_sweeps = 256;
    o->use_graph = 0;
}

void sg_request_default(sg_request *r)
{
    if (!r) return;
    *r = sg_request{};
    r->n_therm = -1;
    r->layout = -1;
    r->exchange_every = 1;
    r->measure_every = 1;
}

sg_status sg_server_create(const sg_server_options *opt, void *stream, sg_server **out)
{
    if (!out) return SG_EINVAL;
    *out = nullptr;
    sg_server *sv = new sg_server();
    if (opt) sv->opt = *opt; else sg_server_options_default(&sv->opt);
    sv->stream = (cudaStream_t)stream;
    if (cudaGetDevice(&sv->device) != cudaSuccess) {
        delete sv;
        return SG_ECUDA;
    }
    if (sv->opt.memory_budget == 0) {
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
            delete sv;
            return SG_ECUDA;
        }
        sv->opt.memory_budget = free_b / 10 * 8;  // leave headroom for other users
    }
    sv->worker = std::thread(worker_loop, sv);
    *out = sv;
    return SG_OK;
}

sg_status sg_server_submit(sg_server *sv, const sg_request *r, int64_t *id_out)
{
    if (!sv || !r || !id_out || !r->T || r->n_T < 1 || r->n_sweeps < 0) return SG_EINVAL;
    Request q;
    q.r = *r;
    q.T.assign(r->T, r->T + r->n_T);
    q.r.T = nullptr;
    q.t_submit = now_s();
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->stop) return SG_EBUSY;
    const int64_t id = sv->next_id++;
    sv->reqs[id] = std::move(q);
    sv->queue.push_back(id);
    *id_out = id;
    sv->cv.notify_all();
    return SG_OK;
}

sg_status sg_server_wait(sg_server *sv, int64_t id, double timeout_s, int *state)
{
    if (!sv) return SG_EINVAL;
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->reqs.find(id);
    if (it == sv->reqs.end()) return SG_EINVAL;
    auto finished = [&] { return sv->reqs[id].state >= RQ_DONE; };
    if (timeout_s < 0) {
        sv->done_cv.wait(lk, finished);
    } else if (!sv->done_cv.wait_for(lk, std::chrono::duration<double>(timeout_s), finished)) {
        if (state) *state = sv->reqs[id].state;
        return SG_ETIMEOUT;
    }
    if (state) *state = sv->reqs[id].state;
    return SG_OK;
}

sg_status sg_server_result(sg_server *sv, int64_t id, double *acc_out, double *latency_s)
{
    if (!sv) return SG_EINVAL;
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->reqs.find(id);
    if (it == sv->reqs.end()) return SG_EINVAL;
    Request &q = it->second;
    if (q.state == RQ_FAILED) return q.err != SG_OK ? q.err : SG_ECUDA;
    if (q.state == RQ_CANCELLED) return SG_ECANCELLED;
    if (q.state != RQ_DONE) return SG_EBUSY;
    if (acc_out) std::copy(q.acc.begin(), q.acc.end(), acc_out);
    if (latency_s) *latency_s = q.t_done - q.t_submit;
    return SG_OK;
}

sg_status sg_server_cancel(sg_server *sv, int64_t id)
{
    if (!sv) return SG_EINVAL;
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->reqs.find(id);
    if (it == sv->reqs.end()) return SG_EINVAL;
    it->second.cancel = true;
    sv->cv.notify_all();
    return SG_OK;
}

sg_status sg_server_release(sg_server *sv, int64_t id)
{
    if (!sv) return SG_EINVAL;
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->reqs.find(id);
    if (it == sv->reqs.end()) return SG_EINVAL;
    if (it->second.state < RQ_DONE) return SG_EBUSY;
    sv->reqs.erase(it);
    return SG_OK;
}

sg_status sg_server_get_stats(sg_server *sv, sg_server_stats *out)
{
    if (!sv || !out) return SG_EINVAL;
    std::lock_guard<std::mutex> lk(sv->mu);
    out->completed = sv->completed;
    out->queued = (int64_t)sv->queue.size();
    out->active = (int64_t)sv->active.size();
    out->rounds = sv->rounds;
    out->attempts = sv->attempts;
    out->busy_seconds = sv->busy_s + (sv->busy_since >= 0 ? now_s() - sv->busy_since : 0.0);
    out->device_bytes_in_use = sv->used;
    out->latency_p50 = percentile(sv->latencies, 0.50);
    out->latency_p99 = percentile(sv->latencies, 0.99);
    return SG_OK;
}

void sg_server_destroy(sg_server *sv)
{
    if (!sv) return;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
        sv->cv.notify_all();
    }
    if (sv->worker.joinable()) sv->worker.join();
    delete sv;
}

}  // extern "C"
