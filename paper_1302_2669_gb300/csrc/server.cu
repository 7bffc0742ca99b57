// Request serving on top of the C ABI: continuous batching of single
// syndromes of mixed code sizes.
//
// The caller submits requests (id, L, sweeps, syndrome bytes) from any
// thread.  A scheduler thread takes the pending requests in arrival order
// into batches of at most max_batch, admits a batch when a slot is free and
// the batch's device scratch fits the memory budget next to the batches in
// flight, and decodes it with surfmcmc_decode_ragged on the slot's own
// context and stream.  Slots run concurrently on the GPU; a batch launches as
// soon as a slot frees up, so requests that arrive while others are on the
// GPU join the next batch.  Finished results (with their latency from
// submission) wait in a queue that the caller polls.  The randomness of a
// request is keyed by its id, so its result does not depend on its batch.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "common.cuh"
#include "surfmcmc.h"

using namespace surfmcmc;

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    uint32_t id;
    int32_t L;
    uint32_t sweeps;
    std::vector<uint8_t> syndrome;
    Clock::time_point t_submit;
};

struct Result {
    uint32_t id;
    int32_t cls;
    uint64_t sum[4];
    double latency_us;
};

struct Slot {
    surfmcmc_ctx* ctx = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    bool busy = false;
    size_t scratch = 0;                  // bytes charged to the memory budget
    std::vector<Request> reqs;           // the batch in flight
    // pinned host staging
    uint8_t* h_syn = nullptr;
    int32_t* h_L = nullptr;
    uint32_t* h_sw = nullptr;
    uint32_t* h_ids = nullptr;
    int32_t* h_cls = nullptr;
    uint64_t* h_sum = nullptr;
    // device outputs
    int32_t* d_cls = nullptr;
    uint64_t* d_sum = nullptr;
};

}  // namespace

struct surfmcmc_server {
    int device = 0;
    double p = 0.1;
    surfmcmc_opts opts;
    uint64_t seed = 0;
    surfmcmc_server_opts sopts;
    std::vector<Slot> slots;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request> pending;
    std::deque<Result> results;
    bool stop = false;
    std::thread worker;
    int64_t admitted = 0, batches = 0, memory_stalls = 0;
    bool waiting_for_memory = false;     // admission is waiting for memory now
    size_t in_flight_bytes = 0;
    std::string error;
};

namespace {

// Device scratch of a ragged batch (upper bound, as the library carves it):
// a fixed part plus, per request, its row, table entries, pure error, sums
// and bundle state.
constexpr size_t kBatchBaseBytes = 64 * 1024;

size_t request_bytes(int L, int R) {
    const size_t nq = (size_t)n_qubits(L), W = (size_t)n_words(L);
    return (size_t)n_stabs(L) + 64 + 2 * W * 4 + (size_t)4 * R * 8 + 2 * nq * 4 + 256;
}

void finish_slot(surfmcmc_server* s, Slot& sl) {
    const Clock::time_point now = Clock::now();
    std::lock_guard<std::mutex> lk(s->mu);
    for (size_t i = 0; i < sl.reqs.size(); ++i) {
        Result r;
        r.id = sl.reqs[i].id;
        r.cls = sl.h_cls[i];
        memcpy(r.sum, sl.h_sum + 4 * i, sizeof r.sum);
        r.latency_us = std::chrono::duration<double, std::micro>(now - sl.reqs[i].t_submit).count();
        s->results.push_back(r);
    }
    sl.reqs.clear();
    sl.busy = false;
    s->in_flight_bytes -= sl.scratch;
    sl.scratch = 0;
    s->cv_done.notify_all();
}

void worker_main(surfmcmc_server* s) {
    cudaSetDevice(s->device);
    const int R = s->opts.chains_per_class;
    for (;;) {
        // retire finished batches
        for (Slot& sl : s->slots)
            if (sl.busy && cudaEventQuery(sl.done) == cudaSuccess) finish_slot(s, sl);
        std::vector<Request> batch;
        Slot* free_slot = nullptr;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            if (s->stop && s->pending.empty()) {
                bool any_busy = false;
                for (Slot& sl : s->slots) any_busy |= sl.busy;
                if (!any_busy) return;
            }
            for (Slot& sl : s->slots)
                if (!sl.busy) {
                    free_slot = &sl;
                    break;
                }
            if (free_slot && !s->pending.empty()) {
                // a partial batch waits up to max_wait_us for company
                const double waited = std::chrono::duration<double, std::micro>(
                                          Clock::now() - s->pending.front().t_submit).count();
                const bool full = (int64_t)s->pending.size() >= s->sopts.max_batch;
                if (full || waited >= s->sopts.max_wait_us || s->stop) {
                    // the batch: the longest prefix of the queue of at most
                    // max_batch requests whose scratch fits the memory budget
                    // next to the batches in flight (at least one request)
                    const size_t budget = (size_t)s->sopts.memory_budget;
                    size_t need = kBatchBaseBytes;
                    int64_t k = 0;
                    for (auto it = s->pending.begin(); it != s->pending.end() && k < s->sopts.max_batch; ++it) {
                        const size_t b = request_bytes(it->L, R);
                        if (budget > 0 && k > 0 && s->in_flight_bytes + need + b > budget) break;
                        need += b;
                        ++k;
                    }
                    if (budget > 0 && s->in_flight_bytes > 0 && s->in_flight_bytes + need > budget) {
                        // not even one request fits: wait for a batch in flight
                        // to finish (counted once per wait)
                        if (!s->waiting_for_memory) ++s->memory_stalls;
                        s->waiting_for_memory = true;
                    } else {
                        s->waiting_for_memory = false;
                        batch.reserve((size_t)k);
                        for (int64_t i = 0; i < k; ++i) {
                            batch.push_back(std::move(s->pending.front()));
                            s->pending.pop_front();
                        }
                        free_slot->scratch = need;
                        s->in_flight_bytes += need;
                        s->admitted += k;
                        ++s->batches;
                    }
                }
            }
            if (batch.empty()) {
                bool any_busy = false;
                for (Slot& sl : s->slots) any_busy |= sl.busy;
                // sleep briefly while batches run; block when idle
                if (any_busy || !s->pending.empty())
                    s->cv_work.wait_for(lk, std::chrono::microseconds(50));
                else
                    s->cv_work.wait_for(lk, std::chrono::milliseconds(5));
                continue;
            }
        }
        // stage and launch the batch on the free slot
        Slot& sl = *free_slot;
        size_t off = 0;
        for (size_t i = 0; i < batch.size(); ++i) {
            memcpy(sl.h_syn + off, batch[i].syndrome.data(), batch[i].syndrome.size());
            off += batch[i].syndrome.size();
            sl.h_L[i] = batch[i].L;
            sl.h_sw[i] = batch[i].sweeps;
            sl.h_ids[i] = batch[i].id;
        }
        const int64_t n = (int64_t)batch.size();
        int rc = surfmcmc_decode_ragged(sl.ctx, sl.h_syn, sl.h_L, sl.h_sw, n, s->p, &s->opts, s->seed, sl.h_ids, 0,
                                        sl.d_cls, sl.d_sum, nullptr, sl.stream);
        if (rc == SURFMCMC_OK) {
            cudaMemcpyAsync(sl.h_cls, sl.d_cls, n * 4, cudaMemcpyDeviceToHost, sl.stream);
            cudaMemcpyAsync(sl.h_sum, sl.d_sum, n * 32, cudaMemcpyDeviceToHost, sl.stream);
            cudaEventRecord(sl.done, sl.stream);
            sl.reqs = std::move(batch);
            sl.busy = true;
        } else {
            std::lock_guard<std::mutex> lk(s->mu);
            s->error = surfmcmc_last_error(sl.ctx);
            const Clock::time_point now = Clock::now();
            for (Request& r : batch) {
                Result res;
                res.id = r.id;
                res.cls = rc;  // negative: the error code
                memset(res.sum, 0, sizeof res.sum);
                res.latency_us = std::chrono::duration<double, std::micro>(now - r.t_submit).count();
                s->results.push_back(res);
            }
            s->in_flight_bytes -= sl.scratch;
            sl.scratch = 0;
            s->cv_done.notify_all();
        }
    }
}

void free_slot_memory(Slot& sl) {
    if (sl.h_syn) cudaFreeHost(sl.h_syn);
    if (sl.h_L) cudaFreeHost(sl.h_L);
    if (sl.h_sw) cudaFreeHost(sl.h_sw);
    if (sl.h_ids) cudaFreeHost(sl.h_ids);
    if (sl.h_cls) cudaFreeHost(sl.h_cls);
    if (sl.h_sum) cudaFreeHost(sl.h_sum);
    if (sl.d_cls) cudaFree(sl.d_cls);
    if (sl.d_sum) cudaFree(sl.d_sum);
    if (sl.done) cudaEventDestroy(sl.done);
    if (sl.stream) cudaStreamDestroy(sl.stream);
    if (sl.ctx) surfmcmc_destroy(sl.ctx);
}

}  // namespace

extern "C" {

void surfmcmc_server_default_opts(surfmcmc_server_opts* o) {
    if (!o) return;
    o->max_batch = 256;
    o->slots = 4;
    o->max_L = SURFMCMC_MAX_L;
    o->memory_budget = 0;
    o->max_wait_us = 200.0;
}

int surfmcmc_server_create(int device, double p, const surfmcmc_opts* opts, uint64_t seed,
                           const surfmcmc_server_opts* sopts_in, surfmcmc_server** out) {
    if (!out) return SURFMCMC_EINVAL;
    *out = nullptr;
    surfmcmc_server_opts so;
    surfmcmc_server_default_opts(&so);
    if (sopts_in) so = *sopts_in;
    if (so.max_batch < 1 || so.slots < 1 || so.slots > 64 || so.max_L < 2 || so.max_L > SURFMCMC_MAX_L ||
        so.memory_budget < 0 || !(so.max_wait_us >= 0.0) || !(p > 0.0 && p <= 0.75))
        return SURFMCMC_EINVAL;
    surfmcmc_server* s = new surfmcmc_server;
    s->device = device;
    s->p = p;
    surfmcmc_default_opts(&s->opts);
    if (opts) s->opts = *opts;
    s->seed = seed;
    s->sopts = so;
    s->slots.resize(so.slots);
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(device);
    int rc = SURFMCMC_OK;
    const size_t row = (size_t)n_stabs(so.max_L);
    for (Slot& sl : s->slots) {
        if ((rc = surfmcmc_create(&sl.ctx, device)) != SURFMCMC_OK) break;
        bool ok = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) == cudaSuccess &&
                  cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) == cudaSuccess &&
                  cudaMallocHost(&sl.h_syn, row * so.max_batch) == cudaSuccess &&
                  cudaMallocHost(&sl.h_L, 4 * so.max_batch) == cudaSuccess &&
                  cudaMallocHost(&sl.h_sw, 4 * so.max_batch) == cudaSuccess &&
                  cudaMallocHost(&sl.h_ids, 4 * so.max_batch) == cudaSuccess &&
                  cudaMallocHost(&sl.h_cls, 4 * so.max_batch) == cudaSuccess &&
                  cudaMallocHost(&sl.h_sum, 32 * so.max_batch) == cudaSuccess &&
                  cudaMalloc(&sl.d_cls, 4 * so.max_batch) == cudaSuccess &&
                  cudaMalloc(&sl.d_sum, 32 * so.max_batch) == cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            rc = SURFMCMC_ENOMEM;
            break;
        }
        // size the slot's scratch once for a full batch of the largest codes,
        // so that no allocation happens while serving
        for (int64_t i = 0; i < so.max_batch; ++i) {
            sl.h_L[i] = so.max_L;
            sl.h_sw[i] = 1;
            sl.h_ids[i] = (uint32_t)i;
        }
        memset(sl.h_syn, 0, row * so.max_batch);
        surfmcmc_opts warm = s->opts;
        warm.n_sweeps = 1;
        warm.burn_in = 0;
        warm.anneal_stages = 0;
        rc = surfmcmc_decode_ragged(sl.ctx, sl.h_syn, sl.h_L, sl.h_sw, so.max_batch, p, &warm, 0, sl.h_ids, 0, sl.d_cls,
                                    sl.d_sum, nullptr, sl.stream);
        if (rc == SURFMCMC_OK && cudaStreamSynchronize(sl.stream) != cudaSuccess) rc = SURFMCMC_ECUDA;
        if (rc != SURFMCMC_OK) break;
    }
    cudaSetDevice(prev);
    if (rc != SURFMCMC_OK) {
        for (Slot& sl : s->slots) free_slot_memory(sl);
        delete s;
        return rc;
    }
    s->worker = std::thread(worker_main, s);
    *out = s;
    return SURFMCMC_OK;
}

int surfmcmc_server_submit(surfmcmc_server* s, uint32_t request_id, int32_t L, uint32_t n_sweeps,
                           const uint8_t* syndrome) {
    if (!s || !syndrome || L < 2 || L > s->sopts.max_L || n_sweeps < 1) return SURFMCMC_EINVAL;
    if (s->opts.n_sweeps && s->opts.anneal_stages > 0 &&
        (uint64_t)n_sweeps * s->opts.burn_in / s->opts.n_sweeps < (uint64_t)s->opts.anneal_stages)
        return SURFMCMC_EINVAL;
    Request r;
    r.id = request_id;
    r.L = L;
    r.sweeps = n_sweeps;
    r.syndrome.assign(syndrome, syndrome + n_stabs(L));
    r.t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) return SURFMCMC_EINVAL;
        s->pending.push_back(std::move(r));
    }
    s->cv_work.notify_one();
    return SURFMCMC_OK;
}

int surfmcmc_server_poll(surfmcmc_server* s, int64_t max_results, uint32_t* ids, int32_t* classes,
                         uint64_t* class_sums, double* latency_us, int64_t* n_out, int32_t wait_us) {
    if (!s || !n_out || max_results < 0 || (max_results > 0 && (!ids || !classes))) return SURFMCMC_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->results.empty() && wait_us > 0)
        s->cv_done.wait_for(lk, std::chrono::microseconds(wait_us), [&] { return !s->results.empty(); });
    int64_t k = 0;
    while (k < max_results && !s->results.empty()) {
        const Result& r = s->results.front();
        ids[k] = r.id;
        classes[k] = r.cls;
        if (class_sums) memcpy(class_sums + 4 * k, r.sum, sizeof r.sum);
        if (latency_us) latency_us[k] = r.latency_us;
        s->results.pop_front();
        ++k;
    }
    *n_out = k;
    return SURFMCMC_OK;
}

int surfmcmc_server_stats(surfmcmc_server* s, int64_t* admitted, int64_t* batches, int64_t* memory_stalls,
                          int64_t* pending) {
    if (!s) return SURFMCMC_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    if (admitted) *admitted = s->admitted;
    if (batches) *batches = s->batches;
    if (memory_stalls) *memory_stalls = s->memory_stalls;
    if (pending) *pending = (int64_t)s->pending.size();
    return SURFMCMC_OK;
}

void surfmcmc_server_destroy(surfmcmc_server* s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(s->device);
    for (Slot& sl : s->slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        free_slot_memory(sl);
    }
    cudaSetDevice(prev);
    delete s;
}

}  // extern "C"
