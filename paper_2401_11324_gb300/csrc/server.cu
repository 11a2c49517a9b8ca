// Serving loop with continuous batching over the batched search.
//
// Requests (host queries with their own k and L) are queued by
// bang_server_submit.  A dispatcher thread owns `streams` slots; each slot has
// page-locked host buffers and device buffers for up to `max_batch` queries,
// allocated once at start, so admission is by device memory: a request waits
// until a slot is free.  When a slot frees, the dispatcher packs as many
// pending requests as fit into one bang_search_batched launch on that slot's
// stream (H2D copy, search, D2H copy, event).  Launches on different slots
// overlap on the GPU, so requests that arrive while others are being searched
// start as soon as a slot frees, not when the whole GPU is idle.  A host
// function enqueued behind each launch's result copies wakes the dispatcher
// when the launch is done (it sleeps otherwise; its events are checked again
// every 2 ms in case a wake-up is missed); results are scattered to the
// requests and their latency (submit to results in host memory) recorded.
#include <cuda_runtime.h>

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

#include "bang.h"
#include "bang_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t ticket = 0;
    uint32_t nq = 0;
    std::vector<unsigned char> queries;
    std::vector<uint32_t> k, L;
    std::vector<uint32_t> ids;
    std::vector<float> dist;
    Clock::time_point t_submit, t_done;
    bool done = false;
    int status = BANG_OK;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    unsigned char *h_q = nullptr;
    uint32_t *h_k = nullptr, *h_L = nullptr, *h_ids = nullptr;
    float *h_dist = nullptr;
    void *d_q = nullptr;
    uint32_t *d_k = nullptr, *d_L = nullptr, *d_ids = nullptr;
    float *d_dist = nullptr;
    std::vector<std::shared_ptr<Request>> batch;
    bool busy = false;
    bang_server *srv = nullptr;     // for the completion host function
};

}  // namespace

struct bang_server {
    bang_index *ix = nullptr;
    bang_server_config cfg{};
    uint32_t d = 0;
    size_t esz = 1;
    int device = 0;
    std::vector<Slot> slots;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<Request>> pending;
    std::unordered_map<uint64_t, std::shared_ptr<Request>> live;
    uint64_t next_ticket = 1;
    bool stopping = false;
    std::thread dispatcher;
    std::string error;
};

namespace {

int sfail(int code, const std::string &msg)
{
    bang::set_error(msg);
    return code;
}

void release_slots(bang_server *s)
{
    for (Slot &sl : s->slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.stream) cudaStreamDestroy(sl.stream);
        cudaFreeHost(sl.h_q); cudaFreeHost(sl.h_k); cudaFreeHost(sl.h_L);
        cudaFreeHost(sl.h_ids); cudaFreeHost(sl.h_dist);
        cudaFree(sl.d_q); cudaFree(sl.d_k); cudaFree(sl.d_L); cudaFree(sl.d_ids); cudaFree(sl.d_dist);
    }
    s->slots.clear();
}

// Runs on a CUDA-owned thread once a slot's launch and result copies are
// done: wake the dispatcher (no CUDA calls are allowed here).
void CUDART_CB slot_done(void *arg)
{
    bang_server *s = static_cast<Slot *>(arg)->srv;
    { std::lock_guard<std::mutex> lk(s->mu); }
    s->cv_work.notify_one();
}

// Launch the packed batch of a slot (called by the dispatcher, lock not held).
int launch_slot(bang_server *s, Slot &sl)
{
    uint32_t nq = 0;
    for (auto &r : sl.batch) {
        std::memcpy(sl.h_q + (size_t)nq * s->d * s->esz, r->queries.data(), r->queries.size());
        std::memcpy(sl.h_k + nq, r->k.data(), r->nq * 4);
        std::memcpy(sl.h_L + nq, r->L.data(), r->nq * 4);
        nq += r->nq;
    }
    const size_t qb = (size_t)nq * s->d * s->esz;
    cudaMemcpyAsync(sl.d_q, sl.h_q, qb, cudaMemcpyHostToDevice, sl.stream);
    cudaMemcpyAsync(sl.d_k, sl.h_k, (size_t)nq * 4, cudaMemcpyHostToDevice, sl.stream);
    cudaMemcpyAsync(sl.d_L, sl.h_L, (size_t)nq * 4, cudaMemcpyHostToDevice, sl.stream);
    bang_search_params p;
    std::memset(&p, 0, sizeof p);
    p.mode = s->cfg.mode;
    p.bloom_log2 = s->cfg.bloom_log2;
    int rc = bang_search_batched(s->ix, sl.d_q, nq, sl.d_k, sl.d_L, s->cfg.k_max, s->cfg.L_max, &p,
                                 sl.d_ids, sl.d_dist, sl.stream);
    if (rc != BANG_OK) return rc;
    const size_t rb = (size_t)nq * s->cfg.k_max * 4;
    cudaMemcpyAsync(sl.h_ids, sl.d_ids, rb, cudaMemcpyDeviceToHost, sl.stream);
    cudaMemcpyAsync(sl.h_dist, sl.d_dist, rb, cudaMemcpyDeviceToHost, sl.stream);
    cudaEventRecord(sl.done, sl.stream);
    cudaLaunchHostFunc(sl.stream, slot_done, &sl);
    return cudaGetLastError() == cudaSuccess ? BANG_OK : BANG_ECUDA;
}

void finish_slot(bang_server *s, Slot &sl, int status)
{
    const auto now = Clock::now();
    uint32_t off = 0;
    const uint32_t km = s->cfg.k_max;
    for (auto &r : sl.batch) {
        r->ids.assign(sl.h_ids + (size_t)off * km, sl.h_ids + (size_t)(off + r->nq) * km);
        r->dist.assign(sl.h_dist + (size_t)off * km, sl.h_dist + (size_t)(off + r->nq) * km);
        off += r->nq;
        r->t_done = now;
        r->status = status;
        r->done = true;
    }
    sl.batch.clear();
    sl.busy = false;
}

void dispatch_loop(bang_server *s)
{
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (true) {
        bool progressed = false;
        // completions
        for (Slot &sl : s->slots) {
            if (!sl.busy) continue;
            cudaError_t q = cudaEventQuery(sl.done);
            if (q == cudaErrorNotReady) continue;
            finish_slot(s, sl, q == cudaSuccess ? BANG_OK : BANG_ECUDA);
            progressed = true;
        }
        if (progressed) s->cv_done.notify_all();
        // admissions: fill every free slot from the pending queue
        for (Slot &sl : s->slots) {
            if (sl.busy || s->pending.empty()) continue;
            uint32_t nq = 0;
            while (!s->pending.empty() && nq + s->pending.front()->nq <= s->cfg.max_batch) {
                nq += s->pending.front()->nq;
                sl.batch.push_back(s->pending.front());
                s->pending.pop_front();
            }
            if (sl.batch.empty()) continue;
            sl.busy = true;
            lk.unlock();
            int rc = launch_slot(s, sl);
            lk.lock();
            if (rc != BANG_OK) finish_slot(s, sl, rc);
            progressed = true;
        }
        bool any_busy = false;
        for (Slot &sl : s->slots) any_busy |= sl.busy;
        if (s->stopping && !any_busy && s->pending.empty()) break;
        if (!progressed) s->cv_work.wait_for(lk, std::chrono::milliseconds(any_busy ? 2 : 5));
    }
}

}  // namespace

extern "C" {

int bang_server_start(bang_index *ix, const bang_server_config *cfg, bang_server **out)
{
    if (!ix || !cfg || !out) return sfail(BANG_EINVAL, "bang_server_start: NULL argument");
    *out = nullptr;
    uint32_t d = 0;
    int32_t dtype = 0;
    if (bang_index_info(ix, nullptr, &d, nullptr, nullptr, &dtype) != BANG_OK || d == 0)
        return sfail(BANG_ESTATE, "bang_server_start: load the index first");
    if (cfg->streams == 0 || cfg->streams > 16)
        return sfail(BANG_EINVAL, "bang_server_start: streams must be 1..16");
    if (cfg->max_batch == 0 || cfg->k_max == 0 || cfg->L_max < cfg->k_max)
        return sfail(BANG_EINVAL, "bang_server_start: need max_batch > 0 and 1 <= k_max <= L_max");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return sfail(BANG_ECUDA, "bang_server_start: no device");
    std::unique_ptr<bang_server> s(new bang_server());
    s->ix = ix;
    s->cfg = *cfg;
    s->d = d;
    s->esz = dtype == BANG_F32 ? 4 : 1;
    s->device = dev;
    s->slots.resize(cfg->streams);
    const size_t nb = cfg->max_batch, km = cfg->k_max;
    for (Slot &sl : s->slots) {
        sl.srv = s.get();
        bool ok = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) == cudaSuccess &&
                  cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) == cudaSuccess &&
                  cudaHostAlloc((void **)&sl.h_q, nb * d * s->esz, 0) == cudaSuccess &&
                  cudaHostAlloc((void **)&sl.h_k, nb * 4, 0) == cudaSuccess &&
                  cudaHostAlloc((void **)&sl.h_L, nb * 4, 0) == cudaSuccess &&
                  cudaHostAlloc((void **)&sl.h_ids, nb * km * 4, 0) == cudaSuccess &&
                  cudaHostAlloc((void **)&sl.h_dist, nb * km * 4, 0) == cudaSuccess &&
                  cudaMalloc(&sl.d_q, nb * d * s->esz) == cudaSuccess &&
                  cudaMalloc((void **)&sl.d_k, nb * 4) == cudaSuccess &&
                  cudaMalloc((void **)&sl.d_L, nb * 4) == cudaSuccess &&
                  cudaMalloc((void **)&sl.d_ids, nb * km * 4) == cudaSuccess &&
                  cudaMalloc((void **)&sl.d_dist, nb * km * 4) == cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            release_slots(s.get());
            return sfail(BANG_ENOMEM, "bang_server_start: slot buffers do not fit; reduce streams or max_batch");
        }
        // one empty launch per stream allocates its work counter up front
        std::fill(sl.h_k, sl.h_k + 1, 1u);
        std::fill(sl.h_L, sl.h_L + 1, cfg->k_max);
        cudaMemset(sl.d_q, 0, d * s->esz);
        cudaMemcpy(sl.d_k, sl.h_k, 4, cudaMemcpyHostToDevice);
        cudaMemcpy(sl.d_L, sl.h_L, 4, cudaMemcpyHostToDevice);
        bang_search_params p;
        std::memset(&p, 0, sizeof p);
        p.mode = cfg->mode;
        p.bloom_log2 = cfg->bloom_log2;
        int rc = bang_search_batched(ix, sl.d_q, 1, sl.d_k, sl.d_L, cfg->k_max, cfg->L_max, &p, sl.d_ids,
                                     sl.d_dist, sl.stream);
        if (rc != BANG_OK || cudaStreamSynchronize(sl.stream) != cudaSuccess) {
            std::string m = std::string("bang_server_start: warm-up search failed: ") + bang_last_error();
            release_slots(s.get());
            return sfail(rc != BANG_OK ? rc : BANG_ECUDA, m);
        }
    }
    bang_server *raw = s.release();
    raw->dispatcher = std::thread(dispatch_loop, raw);
    *out = raw;
    return BANG_OK;
}

int bang_server_submit(bang_server *s, const void *queries, uint32_t nq, const uint32_t *k_per_q,
                       const uint32_t *L_per_q, uint64_t *ticket)
{
    if (!s || !queries || !k_per_q || !L_per_q || !ticket)
        return sfail(BANG_EINVAL, "bang_server_submit: NULL argument");
    if (nq == 0 || nq > s->cfg.max_batch)
        return sfail(BANG_EINVAL, "bang_server_submit: nq must be 1..max_batch");
    auto r = std::make_shared<Request>();
    r->nq = nq;
    const auto *qb = static_cast<const unsigned char *>(queries);
    r->queries.assign(qb, qb + (size_t)nq * s->d * s->esz);
    r->k.assign(k_per_q, k_per_q + nq);
    r->L.assign(L_per_q, L_per_q + nq);
    r->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stopping) return sfail(BANG_ESTATE, "bang_server_submit: server is stopping");
        r->ticket = s->next_ticket++;
        s->live[r->ticket] = r;
        s->pending.push_back(r);
    }
    s->cv_work.notify_one();
    *ticket = r->ticket;
    return BANG_OK;
}

int bang_server_wait(bang_server *s, uint64_t ticket, int32_t timeout_ms, uint32_t *out_ids,
                     float *out_dist, double *latency_ms)
{
    if (!s) return sfail(BANG_EINVAL, "bang_server_wait: NULL server");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->live.find(ticket);
    if (it == s->live.end()) return sfail(BANG_EINVAL, "bang_server_wait: unknown ticket");
    std::shared_ptr<Request> r = it->second;
    auto ready = [&] { return r->done; };
    if (timeout_ms < 0) s->cv_done.wait(lk, ready);
    else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready))
        return sfail(BANG_ETIMEOUT, "bang_server_wait: request not finished in time");
    s->live.erase(it);
    lk.unlock();
    if (r->status != BANG_OK) return sfail(r->status, "bang_server_wait: the batch failed");
    if (out_ids) std::memcpy(out_ids, r->ids.data(), r->ids.size() * 4);
    if (out_dist) std::memcpy(out_dist, r->dist.data(), r->dist.size() * 4);
    if (latency_ms)
        *latency_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
    return BANG_OK;
}

int bang_server_stop(bang_server *s)
{
    if (!s) return BANG_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stopping = true;
    }
    s->cv_work.notify_all();
    if (s->dispatcher.joinable()) s->dispatcher.join();
    release_slots(s);
    delete s;
    return BANG_OK;
}

}  // extern "C"
