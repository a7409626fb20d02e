// Serving loop for heterodyned likelihoods (the Module 2/3 evaluations of Katz,
// arXiv:2111.01064, Sec. III B-C, served to many concurrent samplers).
//
// Continuous batching on one GPU:
//  - sources (prepared references, Sec. II B summary data) stay resident on the device and
//    are admitted while their device footprint fits the memory budget;
//  - a request (one source, W walkers) is copied at submit (the caller may reuse its buffer)
//    and queued; the worker thread packs queued requests - any mix of sources - into one
//    multi-source heterodyne launch whenever a slot is free.  A slot is a fixed pair of device
//    buffers (theta in, lnL out) inside the budget with its own stream, so a new batch's
//    copies and kernel overlap the batches already in flight;
//  - completion is signalled from the stream (cudaLaunchHostFunc); the worker scatters the
//    results into the requests' output buffers and wakes the waiters;
//  - per-request latency (submit -> results written) feeds the p50/p99 statistics.
// A walker's lnL does not depend on the batch it was packed into (fixed-order per-walker
// computation), so a request gives the same result alone and in the mix.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <random>
#include <thread>
#include <unordered_map>
#include <vector>

#include "mbh_internal.cuh"
#include "mbh_model.cuh"

using namespace mbh;
using Clock = std::chrono::steady_clock;

namespace {

struct Request {
    uint64_t id = 0;
    int32_t source = -1;
    int64_t W = 0;
    std::vector<double> theta;   // [11][W], pinned-staged at launch
    double* out_host = nullptr;  // caller's [3][W]
    Clock::time_point t_submit, t_done;
    mbh_status status = MBH_OK;
    bool done = false;
    bool launched = false;
};

struct Source {
    const mbh_ref* ref = nullptr;
    size_t bytes = 0;
    int64_t pending = 0;   // requests queued or in flight
    int64_t inflight = 0;  // requests in batches on the GPU (using `ref`)
};

struct Slot {
    mbh_server* owner = nullptr;   // for the completion callback
    cudaStream_t stream = nullptr;
    double* theta_dev = nullptr;   // [11][max_batch]
    double* out_dev = nullptr;     // [3][max_batch]
    double* theta_host = nullptr;  // pinned
    double* out_host = nullptr;    // pinned
    std::vector<std::shared_ptr<Request>> reqs;
    int64_t W = 0;
    bool busy = false;
    std::atomic<bool> finished{false};
};

size_t ref_bytes(const mbh_ref* R)
{
    const size_t E = (size_t)R->E;
    size_t b = E * (18 * sizeof(double) + sizeof(double) + sizeof(MixBin)) +
               (E + 1) * (sizeof(int64_t) + sizeof(double) + 2 * 3 * sizeof(double2) + sizeof(MixEdge)) +
               11 * sizeof(double) + 2 * sizeof(double);
    if (R->modes != 1u)   // per-mode reference tables of a higher-mode reference
        b += (E + 1) * (kHmModes * sizeof(MixModeHM) + 3 * sizeof(float2));
    return b;
}

}  // namespace

struct mbh_server {
    mbh_server_opts opts{};
    int device = 0;
    size_t slot_bytes = 0;
    size_t source_bytes = 0;
    std::vector<std::unique_ptr<Slot>> slots;
    std::unordered_map<int32_t, Source> sources;
    int32_t next_source = 0;
    uint64_t next_id = 1;
    std::deque<std::shared_ptr<Request>> queue;
    std::unordered_map<uint64_t, std::shared_ptr<Request>> live;
    std::mutex mu;
    std::condition_variable cv_work;   // worker: new requests or a finished slot
    std::condition_variable cv_done;   // waiters
    std::thread worker;
    bool stop = false;
    bool paused = false;
    // statistics
    std::vector<double> latencies_ms;
    int64_t completed = 0, walkers_done = 0, batches = 0, batch_walkers = 0, rejected = 0;
    Clock::time_point t_first, t_last;
    bool any = false;
};

namespace {

// Stream callback after a batch's copies and kernel: marks the slot finished and wakes the
// worker (no CUDA calls here).
void CUDART_CB slot_done(void* p)
{
    Slot* sl = static_cast<Slot*>(p);
    sl->finished.store(true, std::memory_order_release);
    {
        std::lock_guard<std::mutex> lk(sl->owner->mu);
    }
    sl->owner->cv_work.notify_one();
}

// Completes the requests of a finished slot (caller holds the lock).
void finish_slot(mbh_server* S, Slot& sl, mbh_status st)
{
    int64_t off = 0;
    const auto now = Clock::now();
    for (auto& r : sl.reqs) {
        if (st == MBH_OK && r->status == MBH_OK) {
            for (int q = 0; q < 3; ++q)
                std::memcpy(r->out_host + (int64_t)q * r->W, sl.out_host + (int64_t)q * sl.W + off,
                            sizeof(double) * r->W);
        } else if (r->status == MBH_OK) {
            r->status = st;
        }
        off += r->W;
        r->t_done = now;
        r->done = true;
        auto it = S->sources.find(r->source);
        if (it != S->sources.end()) {
            --it->second.pending;
            --it->second.inflight;
        }
        if (r->status == MBH_OK) {
            S->latencies_ms.push_back(std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count());
            ++S->completed;
            S->walkers_done += r->W;
            S->t_last = now;
        }
    }
    sl.reqs.clear();
    sl.W = 0;
    sl.busy = false;
    sl.finished.store(false);
    S->cv_done.notify_all();
}

// Packs queued requests into a free slot and launches it (caller holds the lock; the lock is
// released around the host copies and launches).
bool launch_one(mbh_server* S, std::unique_lock<std::mutex>& lk)
{
    Slot* sl = nullptr;
    for (auto& s : S->slots)
        if (!s->busy) {
            sl = s.get();
            break;
        }
    if (!sl || S->queue.empty()) return false;
    // requests of evicted sources fail; the others are packed in arrival order
    std::vector<std::shared_ptr<Request>> batch;
    int64_t W = 0;
    while (!S->queue.empty()) {
        auto& r = S->queue.front();
        if (!S->sources.count(r->source)) {
            r->status = MBH_EINVAL;
            r->done = true;
            r->t_done = Clock::now();
            S->queue.pop_front();
            S->cv_done.notify_all();
            continue;
        }
        if (W + r->W > S->opts.max_batch_walkers) break;
        W += r->W;
        r->launched = true;
        batch.push_back(r);
        S->queue.pop_front();
    }
    if (batch.empty()) return false;
    sl->busy = true;
    sl->reqs = batch;
    sl->W = W;
    std::vector<const mbh_ref*> refs;
    std::vector<int64_t> offsets{0};
    for (auto& r : batch) {
        Source& src = S->sources[r->source];
        refs.push_back(src.ref);
        ++src.inflight;
        offsets.push_back(offsets.back() + r->W);
    }
    ++S->batches;
    S->batch_walkers += W;
    lk.unlock();
    // theta of the batch, SoA [11][W], into the slot's pinned buffer
    int64_t off = 0;
    for (auto& r : batch) {
        for (int j = 0; j < 11; ++j)
            std::memcpy(sl->theta_host + (int64_t)j * W + off, r->theta.data() + (int64_t)j * r->W,
                        sizeof(double) * r->W);
        off += r->W;
    }
    mbh_status st = MBH_OK;
    cudaError_t e = cudaMemcpyAsync(sl->theta_dev, sl->theta_host, sizeof(double) * 11 * W,
                                    cudaMemcpyHostToDevice, sl->stream);
    if (e != cudaSuccess) st = cuda_fail(e, "server H2D");
    if (st == MBH_OK) {
        const mbh_het_config* cfg = S->opts.config.threads_per_walker > 0 ? &S->opts.config : nullptr;
        st = het_loglike_batch_cfg(refs.data(), offsets.data(), (int32_t)refs.size(), sl->theta_dev,
                                   S->opts.precision, cfg, sl->out_dev, sl->stream);
    }
    if (st == MBH_OK) {
        e = cudaMemcpyAsync(sl->out_host, sl->out_dev, sizeof(double) * 3 * W, cudaMemcpyDeviceToHost,
                            sl->stream);
        if (e != cudaSuccess) st = cuda_fail(e, "server D2H");
    }
    if (st == MBH_OK) {
        e = cudaLaunchHostFunc(sl->stream, slot_done, sl);
        if (e != cudaSuccess) st = cuda_fail(e, "server callback");
    }
    lk.lock();
    if (st != MBH_OK) finish_slot(S, *sl, st);
    return true;
}

void worker_loop(mbh_server* S)
{
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    while (true) {
        for (auto& s : S->slots)
            if (s->busy && s->finished.load(std::memory_order_acquire)) finish_slot(S, *s, MBH_OK);
        bool launched = false;
        if (!S->stop && !S->paused) launched = launch_one(S, lk);
        if (launched) continue;
        bool inflight = false;
        for (auto& s : S->slots) inflight |= s->busy;
        if (S->stop && !inflight) break;
        S->cv_work.wait_for(lk, std::chrono::milliseconds(50));
    }
}

}  // namespace

extern "C" mbh_status mbh_server_create(const mbh_server_opts* opts, mbh_server** out)
{
    if (!opts || !out) return fail(MBH_EINVAL, "NULL argument");
    *out = nullptr;
    if (opts->max_batch_walkers < 1 || opts->max_inflight_batches < 1 || opts->max_queue < 1)
        return fail(MBH_EINVAL, "max_batch_walkers, max_inflight_batches and max_queue must be >= 1");
    if (opts->precision != MBH_FP64 && opts->precision != MBH_MIXED && opts->precision != MBH_MIXED_F32)
        return fail(MBH_EINVAL, "unknown precision");
    if (mbh_status s = check_device()) return s;
    auto S = std::make_unique<mbh_server>();
    S->opts = *opts;
    cudaGetDevice(&S->device);
    S->slot_bytes = sizeof(double) * 14 * (size_t)opts->max_batch_walkers;
    if (S->slot_bytes * opts->max_inflight_batches > (size_t)std::max<int64_t>(0, opts->hbm_budget_bytes))
        return fail(MBH_EBUSY, "slot buffers (%zu bytes) exceed the memory budget (%lld bytes)",
                    S->slot_bytes * opts->max_inflight_batches, (long long)opts->hbm_budget_bytes);
    for (int i = 0; i < opts->max_inflight_batches; ++i) {
        auto sl = std::make_unique<Slot>();
        sl->owner = S.get();
        cudaError_t e = cudaStreamCreateWithFlags(&sl->stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaMalloc(&sl->theta_dev, sizeof(double) * 11 * opts->max_batch_walkers);
        if (e == cudaSuccess) e = cudaMalloc(&sl->out_dev, sizeof(double) * 3 * opts->max_batch_walkers);
        if (e == cudaSuccess) e = cudaMallocHost(&sl->theta_host, sizeof(double) * 11 * opts->max_batch_walkers);
        if (e == cudaSuccess) e = cudaMallocHost(&sl->out_host, sizeof(double) * 3 * opts->max_batch_walkers);
        S->slots.push_back(std::move(sl));
        if (e != cudaSuccess) {
            mbh_server_free(S.release());
            return cuda_fail(e, "mbh_server_create");
        }
    }
    S->worker = std::thread(worker_loop, S.get());
    *out = S.release();
    return MBH_OK;
}

extern "C" mbh_status mbh_server_add_source(mbh_server* S, const mbh_ref* ref, int32_t* source_id)
{
    if (!S || !ref || !source_id) return fail(MBH_EINVAL, "NULL argument");
    if (ref->device != S->device) return fail(MBH_EINVAL, "reference lives on another device");
    std::lock_guard<std::mutex> lk(S->mu);
    const size_t b = ref_bytes(ref);
    const size_t used = S->source_bytes + S->slot_bytes * S->slots.size();
    if (used + b > (size_t)S->opts.hbm_budget_bytes) {
        ++S->rejected;
        return fail(MBH_EBUSY, "source needs %zu bytes; %zu of the %lld-byte budget are in use", b, used,
                    (long long)S->opts.hbm_budget_bytes);
    }
    const int32_t id = S->next_source++;
    S->sources[id] = Source{ref, b, 0};
    S->source_bytes += b;
    *source_id = id;
    return MBH_OK;
}

extern "C" mbh_status mbh_server_remove_source(mbh_server* S, int32_t source_id)
{
    if (!S) return fail(MBH_EINVAL, "NULL server");
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->sources.find(source_id);
    if (it == S->sources.end()) return fail(MBH_EINVAL, "unknown source %d", source_id);
    // queued requests of this source fail with MBH_EINVAL; batches already in flight finish
    // (they hold the reference until then: wait for them before releasing the entry)
    for (auto qi = S->queue.begin(); qi != S->queue.end();) {
        if ((*qi)->source == source_id) {
            (*qi)->status = MBH_EINVAL;
            (*qi)->done = true;
            (*qi)->t_done = Clock::now();
            it->second.pending--;
            qi = S->queue.erase(qi);
        } else {
            ++qi;
        }
    }
    S->cv_done.notify_all();
    S->cv_done.wait(lk, [&] { return S->sources[source_id].pending <= 0; });
    it = S->sources.find(source_id);   // the map may have been rehashed meanwhile
    S->source_bytes -= it->second.bytes;
    S->sources.erase(it);
    return MBH_OK;
}

extern "C" mbh_status mbh_server_replace_source(mbh_server* S, int32_t source_id, const mbh_ref* ref)
{
    if (!S || !ref) return fail(MBH_EINVAL, "NULL argument");
    if (ref->device != S->device) return fail(MBH_EINVAL, "reference lives on another device");
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->sources.find(source_id);
    if (it == S->sources.end()) return fail(MBH_EINVAL, "unknown source %d", source_id);
    const size_t b = ref_bytes(ref);
    const size_t used = S->source_bytes - it->second.bytes + S->slot_bytes * S->slots.size();
    if (used + b > (size_t)S->opts.hbm_budget_bytes) {
        ++S->rejected;
        return fail(MBH_EBUSY, "replacement needs %zu bytes; %zu of the %lld-byte budget are in use", b,
                    used, (long long)S->opts.hbm_budget_bytes);
    }
    // batches launched from now on use the new reference; wait for those in flight on the old
    S->source_bytes += b - it->second.bytes;
    it->second.bytes = b;
    it->second.ref = ref;
    S->cv_done.wait(lk, [&] {
        auto jt = S->sources.find(source_id);
        return jt == S->sources.end() || jt->second.inflight <= 0;
    });
    return MBH_OK;
}

extern "C" mbh_status mbh_server_submit(mbh_server* S, int32_t source_id, const double* theta_host,
                                        int64_t W, double* out_host, uint64_t* request_id)
{
    if (!S || !theta_host || !out_host || !request_id) return fail(MBH_EINVAL, "NULL argument");
    if (W < 1 || W > S->opts.max_batch_walkers)
        return fail(MBH_EINVAL, "W=%lld outside [1, max_batch_walkers=%d]", (long long)W, S->opts.max_batch_walkers);
    auto r = std::make_shared<Request>();
    r->source = source_id;
    r->W = W;
    r->out_host = out_host;
    r->theta.assign(theta_host, theta_host + 11 * W);
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stop) return fail(MBH_EINVAL, "server is shutting down");
    auto it = S->sources.find(source_id);
    if (it == S->sources.end()) return fail(MBH_EINVAL, "unknown source %d", source_id);
    if ((int64_t)S->queue.size() >= S->opts.max_queue) {
        ++S->rejected;
        return fail(MBH_EBUSY, "queue full (%d requests)", S->opts.max_queue);
    }
    r->id = S->next_id++;
    r->t_submit = Clock::now();
    if (!S->any) {
        S->t_first = r->t_submit;
        S->any = true;
    }
    it->second.pending++;
    S->queue.push_back(r);
    S->live[r->id] = r;
    *request_id = r->id;
    S->cv_work.notify_one();
    return MBH_OK;
}

extern "C" mbh_status mbh_server_wait(mbh_server* S, uint64_t request_id, int32_t timeout_ms,
                                      mbh_status* request_status)
{
    if (!S) return fail(MBH_EINVAL, "NULL server");
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->live.find(request_id);
    if (it == S->live.end()) return fail(MBH_EINVAL, "unknown request %llu", (unsigned long long)request_id);
    auto r = it->second;
    bool ok = true;
    if (timeout_ms < 0)
        S->cv_done.wait(lk, [&] { return r->done; });
    else
        ok = S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return r->done; });
    if (!ok) return fail(MBH_ETIMEOUT, "request %llu not done after %d ms", (unsigned long long)request_id, timeout_ms);
    if (request_status) *request_status = r->status;
    S->live.erase(request_id);
    return MBH_OK;
}

extern "C" mbh_status mbh_server_cancel(mbh_server* S, uint64_t request_id)
{
    if (!S) return fail(MBH_EINVAL, "NULL server");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->live.find(request_id);
    if (it == S->live.end()) return fail(MBH_EINVAL, "unknown request %llu", (unsigned long long)request_id);
    auto r = it->second;
    if (r->done || r->launched) return fail(MBH_EBUSY, "request %llu already launched", (unsigned long long)request_id);
    for (auto qi = S->queue.begin(); qi != S->queue.end(); ++qi)
        if ((*qi)->id == request_id) {
            S->queue.erase(qi);
            break;
        }
    r->status = MBH_ECANCELED;
    r->done = true;
    r->t_done = Clock::now();
    auto si = S->sources.find(r->source);
    if (si != S->sources.end()) si->second.pending--;
    S->cv_done.notify_all();
    return MBH_OK;
}

extern "C" mbh_status mbh_server_pause(mbh_server* S, int32_t paused)
{
    if (!S) return fail(MBH_EINVAL, "NULL server");
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->paused = paused != 0;
    }
    S->cv_work.notify_one();
    return MBH_OK;
}

extern "C" mbh_status mbh_server_stats(mbh_server* S, mbh_server_report* out)
{
    if (!S || !out) return fail(MBH_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(S->mu);
    std::memset(out, 0, sizeof *out);
    out->completed = S->completed;
    out->walkers = S->walkers_done;
    out->batches = S->batches;
    out->rejected = S->rejected;
    out->queued = (int64_t)S->queue.size();
    out->mean_batch_walkers = S->batches ? (double)S->batch_walkers / S->batches : 0.0;
    out->source_bytes = (int64_t)S->source_bytes;
    out->slot_bytes = (int64_t)(S->slot_bytes * S->slots.size());
    if (!S->latencies_ms.empty()) {
        std::vector<double> v = S->latencies_ms;
        auto q = [&](double p) {
            const size_t k = std::min(v.size() - 1, (size_t)std::llround(p * (v.size() - 1)));
            std::nth_element(v.begin(), v.begin() + k, v.end());
            return v[k];
        };
        out->p50_ms = q(0.50);
        out->p99_ms = q(0.99);
        out->max_ms = *std::max_element(v.begin(), v.end());
        const double span = std::chrono::duration<double>(S->t_last - S->t_first).count();
        out->walkers_per_s = span > 0 ? S->walkers_done / span : 0.0;
    }
    return MBH_OK;
}

extern "C" mbh_status mbh_server_reset_stats(mbh_server* S)
{
    if (!S) return fail(MBH_EINVAL, "NULL server");
    std::lock_guard<std::mutex> lk(S->mu);
    S->latencies_ms.clear();
    S->completed = S->walkers_done = S->batches = S->batch_walkers = S->rejected = 0;
    S->any = false;
    return MBH_OK;
}

extern "C" void mbh_server_free(mbh_server* S)
{
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        // queued requests that were never launched are cancelled
        for (auto& r : S->queue) {
            r->status = MBH_ECANCELED;
            r->done = true;
        }
        S->queue.clear();
        S->cv_done.notify_all();
    }
    S->cv_work.notify_all();
    if (S->worker.joinable()) S->worker.join();
    for (auto& sl : S->slots) {
        if (sl->stream) cudaStreamSynchronize(sl->stream);
        if (sl->stream) cudaStreamDestroy(sl->stream);
        cudaFree(sl->theta_dev);
        cudaFree(sl->out_dev);
        cudaFreeHost(sl->theta_host);
        cudaFreeHost(sl->out_host);
    }
    delete S;
}

// ------------------------------------------------------------------------------------------
// Load generator: n_clients sampler threads, each submitting requests of its own source at
// Poisson arrival times (open loop: a client does not wait for a result before its next
// arrival), request sizes log-uniform in [min_walkers, max_walkers], walkers taken from the
// client's pool; results are collected as they complete.  The server's statistics are reset
// at the start, so its latency percentiles describe this run.
// ------------------------------------------------------------------------------------------
extern "C" mbh_status mbh_server_loadgen(mbh_server* S, const int32_t* source_ids, int32_t n_clients,
                                         const double* const* pools_host, int64_t pool,
                                         const mbh_loadgen_opts* o, mbh_loadgen_report* out)
{
    if (!S || !source_ids || !pools_host || !o || !out) return fail(MBH_EINVAL, "NULL argument");
    if (n_clients < 1 || pool < 1) return fail(MBH_EINVAL, "need n_clients >= 1 and pool >= 1");
    if (!(o->rate_per_s > 0.0) || !(o->seconds > 0.0)) return fail(MBH_EINVAL, "rate and seconds must be > 0");
    if (o->rate_per_s * o->seconds > 1e7) return fail(MBH_EINVAL, "more than 1e7 arrivals requested");
    if (o->min_walkers < 1 || o->max_walkers < o->min_walkers || o->max_walkers > pool ||
        o->max_walkers > S->opts.max_batch_walkers)
        return fail(MBH_EINVAL, "request sizes must satisfy 1 <= min <= max <= min(pool, max_batch_walkers)");
    for (int32_t c = 0; c < n_clients; ++c)
        if (!pools_host[c]) return fail(MBH_EINVAL, "pool %d is NULL", c);
    mbh_server_reset_stats(S);
    std::atomic<int64_t> submitted{0}, completed{0}, rejected{0}, failed{0}, walkers{0};
    const auto t0 = Clock::now() + std::chrono::milliseconds(5);
    auto client = [&](int32_t c) {
        std::mt19937_64 rng(o->seed * 1000003ull + (uint64_t)c);
        std::exponential_distribution<double> gap(o->rate_per_s / n_clients);
        std::uniform_real_distribution<double> lsz(std::log((double)o->min_walkers), std::log((double)o->max_walkers + 1.0));
        struct Out {
            uint64_t id;
            int64_t W;
            std::vector<double> res;
        };
        std::deque<Out> outstanding;
        std::vector<double> th;
        auto reap = [&](bool block) {
            while (!outstanding.empty()) {
                mbh_status rs = MBH_OK;
                const mbh_status w = mbh_server_wait(S, outstanding.front().id, block ? -1 : 0, &rs);
                if (w == MBH_ETIMEOUT) return;
                if (w == MBH_OK && rs == MBH_OK) {
                    ++completed;
                    walkers += outstanding.front().W;
                } else {
                    ++failed;
                }
                outstanding.pop_front();
            }
        };
        double t = 0.0;
        while (true) {
            t += gap(rng);
            if (t > o->seconds) break;
            const int64_t W = std::min<int64_t>(o->max_walkers, std::max<int64_t>(o->min_walkers, (int64_t)std::exp(lsz(rng))));
            const int64_t off = (int64_t)(rng() % (uint64_t)(pool - W + 1));
            th.resize(11 * W);
            for (int j = 0; j < 11; ++j)
                std::memcpy(th.data() + (int64_t)j * W, pools_host[c] + (int64_t)j * pool + off, sizeof(double) * W);
            std::this_thread::sleep_until(t0 + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(t)));
            Out rec{0, W, std::vector<double>(3 * W)};
            const mbh_status st = mbh_server_submit(S, source_ids[c], th.data(), W, rec.res.data(), &rec.id);
            if (st == MBH_OK) {
                ++submitted;
                outstanding.push_back(std::move(rec));
            } else {
                ++rejected;
            }
            reap(false);
        }
        reap(true);
    };
    std::vector<std::thread> threads;
    for (int32_t c = 0; c < n_clients; ++c) threads.emplace_back(client, c);
    for (auto& th : threads) th.join();
    const double wall = std::chrono::duration<double>(Clock::now() - t0).count();
    mbh_server_report rep{};
    mbh_server_stats(S, &rep);
    std::memset(out, 0, sizeof *out);
    out->offered_per_s = o->rate_per_s;
    out->submitted = submitted.load();
    out->completed = completed.load();
    out->rejected = rejected.load();
    out->failed = failed.load();
    out->wall_seconds = wall;
    out->completed_per_s = completed.load() / wall;
    out->walkers_per_s = walkers.load() / wall;
    out->p50_ms = rep.p50_ms;
    out->p99_ms = rep.p99_ms;
    out->max_ms = rep.max_ms;
    out->batches = rep.batches;
    out->mean_batch_walkers = rep.mean_batch_walkers;
    return MBH_OK;
}
