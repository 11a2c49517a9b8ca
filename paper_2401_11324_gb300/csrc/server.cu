// Serving loop with continuous batching over the batched search.
//
// Requests (host queries with their own k and L) are queued by
// bang_server_submit.  Admission is by device memory: the server owns one
// device arena of `mem_bytes` and a page-locked host mirror of it, allocated
// at start, and every launch takes a contiguous region of both for its batch
// (queries, k, L, result ids and distances), allocated first-in first-out
// and released when the launch's results are on the host.  A dispatcher
// thread packs pending requests, in arrival order, into one
// bang_search_batched launch as soon as a stream is free and the arena has
// room for the batch (at most max_batch queries); a request that does not fit
// waits until earlier launches release their memory.  Launches on different
// streams overlap on the GPU, so requests that arrive while others are being
// searched start as soon as memory and a stream free up.  A host function
// enqueued behind each launch's result copies wakes the dispatcher (it
// sleeps otherwise; its events are checked again every 2 ms in case a wake-up
// is missed); results are scattered to the requests and their latency
// (submit to results in host memory) recorded.
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
constexpr size_t kAlign = 256;

size_t up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

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

// A launch in flight: its arena region and the requests it carries.
struct Launch {
    size_t off = 0, bytes = 0;
    uint32_t nq = 0;
    std::vector<std::shared_ptr<Request>> batch;
    bool finished = false;
};

struct Stream {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    std::shared_ptr<Launch> launch;        // null: free
    bang_server *srv = nullptr;            // for the completion host function
};

}  // namespace

struct bang_server {
    bang_index *ix = nullptr;
    bang_server_config cfg{};
    uint32_t d = 0;
    size_t esz = 1;
    int device = 0;
    size_t cap = 0;                        // arena bytes
    unsigned char *d_arena = nullptr, *h_arena = nullptr;
    std::deque<std::shared_ptr<Launch>> regions;   // live regions in allocation order
    std::vector<Stream> streams;
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

// Arena bytes of a batch of nq queries: queries, k, L, ids, distances.
size_t batch_bytes(const bang_server *s, uint32_t nq)
{
    return up(static_cast<size_t>(nq) * s->d * s->esz) + 2 * up(static_cast<size_t>(nq) * 4) +
           2 * up(static_cast<size_t>(nq) * s->cfg.k_max * 4);
}

// First-in first-out allocation in the arena: after the newest live region,
// or from the start when the space behind it is too short and the oldest
// region leaves room before it.  Returns false when the batch must wait.
bool arena_alloc(const bang_server *s, size_t bytes, size_t &off)
{
    if (bytes > s->cap) return false;
    if (s->regions.empty()) {
        off = 0;
        return true;
    }
    const size_t head = s->regions.front()->off;
    const size_t tail = s->regions.back()->off + s->regions.back()->bytes;
    if (tail > head) {                     // live regions in one piece: [head, tail)
        if (s->cap - tail >= bytes) { off = tail; return true; }
        if (head >= bytes) { off = 0; return true; }
        return false;
    }
    if (head - tail >= bytes) { off = tail; return true; }   // wrapped: free is [tail, head)
    return false;
}

void release_regions(bang_server *s)
{
    while (!s->regions.empty() && s->regions.front()->finished) s->regions.pop_front();
}

// Runs on a CUDA-owned thread once a launch and its result copies are done:
// wake the dispatcher (no CUDA calls are allowed here).
void CUDART_CB launch_done(void *arg)
{
    bang_server *s = static_cast<Stream *>(arg)->srv;
    { std::lock_guard<std::mutex> lk(s->mu); }
    s->cv_work.notify_one();
}

struct Views {
    unsigned char *q;
    uint32_t *k, *L, *ids;
    float *dist;
};

// The buffers of a batch of nq queries inside a region starting at `base`.
Views views(unsigned char *base, const bang_server *s, uint32_t nq)
{
    Views v;
    size_t o = 0;
    v.q = base + o;
    o += up(static_cast<size_t>(nq) * s->d * s->esz);
    v.k = reinterpret_cast<uint32_t *>(base + o);
    o += up(static_cast<size_t>(nq) * 4);
    v.L = reinterpret_cast<uint32_t *>(base + o);
    o += up(static_cast<size_t>(nq) * 4);
    v.ids = reinterpret_cast<uint32_t *>(base + o);
    o += up(static_cast<size_t>(nq) * s->cfg.k_max * 4);
    v.dist = reinterpret_cast<float *>(base + o);
    return v;
}

// Launch a packed batch on a free stream (dispatcher, lock not held).
int start_launch(bang_server *s, Stream &st, Launch &ln)
{
    const Views h = views(s->h_arena + ln.off, s, ln.nq), dv = views(s->d_arena + ln.off, s, ln.nq);
    uint32_t nq = 0;
    for (auto &r : ln.batch) {
        std::memcpy(h.q + static_cast<size_t>(nq) * s->d * s->esz, r->queries.data(), r->queries.size());
        std::memcpy(h.k + nq, r->k.data(), r->nq * 4);
        std::memcpy(h.L + nq, r->L.data(), r->nq * 4);
        nq += r->nq;
    }
    const size_t in_bytes = reinterpret_cast<unsigned char *>(h.ids) - h.q;   // queries, k and L
    cudaMemcpyAsync(dv.q, h.q, in_bytes, cudaMemcpyHostToDevice, st.stream);
    bang_search_params p;
    std::memset(&p, 0, sizeof p);
    p.mode = s->cfg.mode;
    p.bloom_log2 = s->cfg.bloom_log2;
    p.early_codes = s->cfg.early_codes;
    int rc = bang_search_batched(s->ix, dv.q, nq, dv.k, dv.L, s->cfg.k_max, s->cfg.L_max, &p, dv.ids,
                                 dv.dist, st.stream);
    if (rc != BANG_OK) return rc;
    const size_t out_bytes = 2 * up(static_cast<size_t>(nq) * s->cfg.k_max * 4);   // ids, distances
    cudaMemcpyAsync(h.ids, dv.ids, out_bytes, cudaMemcpyDeviceToHost, st.stream);
    cudaEventRecord(st.done, st.stream);
    cudaLaunchHostFunc(st.stream, launch_done, &st);
    return cudaGetLastError() == cudaSuccess ? BANG_OK : BANG_ECUDA;
}

// Results of a finished launch to its requests, then its region released
// (lock held).
void finish_launch(bang_server *s, Stream &st, int status)
{
    Launch &ln = *st.launch;
    const Views h = views(s->h_arena + ln.off, s, ln.nq);
    const auto now = Clock::now();
    uint32_t off = 0;
    const uint32_t km = s->cfg.k_max;
    for (auto &r : ln.batch) {
        r->ids.assign(h.ids + static_cast<size_t>(off) * km, h.ids + static_cast<size_t>(off + r->nq) * km);
        r->dist.assign(h.dist + static_cast<size_t>(off) * km, h.dist + static_cast<size_t>(off + r->nq) * km);
        off += r->nq;
        r->t_done = now;
        r->status = status;
        r->done = true;
    }
    ln.batch.clear();
    ln.finished = true;
    st.launch.reset();
    release_regions(s);
}

void dispatch_loop(bang_server *s)
{
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (true) {
        bool progressed = false;
        for (Stream &st : s->streams) {            // completions
            if (!st.launch) continue;
            cudaError_t q = cudaEventQuery(st.done);
            if (q == cudaErrorNotReady) continue;
            finish_launch(s, st, q == cudaSuccess ? BANG_OK : BANG_ECUDA);
            progressed = true;
        }
        if (progressed) s->cv_done.notify_all();
        // admissions: pending requests in arrival order, as memory allows
        for (Stream &st : s->streams) {
            if (st.launch || s->pending.empty()) continue;
            auto ln = std::make_shared<Launch>();
            uint32_t nq = 0;
            size_t off = 0;
            while (!s->pending.empty() && nq + s->pending.front()->nq <= s->cfg.max_batch) {
                size_t o2 = 0;
                if (!arena_alloc(s, batch_bytes(s, nq + s->pending.front()->nq), o2)) break;
                off = o2;
                nq += s->pending.front()->nq;
                ln->batch.push_back(s->pending.front());
                s->pending.pop_front();
            }
            if (nq == 0) break;                    // memory full: wait for a release
            ln->off = off;
            ln->nq = nq;
            ln->bytes = batch_bytes(s, nq);
            s->regions.push_back(ln);
            st.launch = ln;
            lk.unlock();
            int rc = start_launch(s, st, *ln);
            lk.lock();
            if (rc != BANG_OK) finish_launch(s, st, rc);
            progressed = true;
        }
        bool any_busy = false;
        for (Stream &st : s->streams) any_busy |= static_cast<bool>(st.launch);
        if (s->stopping && !any_busy && s->pending.empty()) break;
        if (!progressed) s->cv_work.wait_for(lk, std::chrono::milliseconds(any_busy ? 2 : 5));
    }
}

void release_all(bang_server *s)
{
    for (Stream &st : s->streams) {
        if (st.stream) cudaStreamSynchronize(st.stream);
        if (st.done) cudaEventDestroy(st.done);
        if (st.stream) cudaStreamDestroy(st.stream);
    }
    s->streams.clear();
    if (s->d_arena) cudaFree(s->d_arena);
    if (s->h_arena) cudaFreeHost(s->h_arena);
    s->d_arena = s->h_arena = nullptr;
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
    s->cap = cfg->mem_bytes ? static_cast<size_t>(cfg->mem_bytes)
                            : cfg->streams * batch_bytes(s.get(), cfg->max_batch);
    if (s->cap < batch_bytes(s.get(), 1))
        return sfail(BANG_EINVAL, "bang_server_start: mem_bytes holds not even one query");
    if (cudaMalloc(&s->d_arena, s->cap) != cudaSuccess || cudaHostAlloc(&s->h_arena, s->cap, 0) != cudaSuccess) {
        cudaGetLastError();
        release_all(s.get());
        return sfail(BANG_ENOMEM, "bang_server_start: the arena does not fit; lower mem_bytes");
    }
    s->streams.resize(cfg->streams);
    for (Stream &st : s->streams) {
        st.srv = s.get();
        if (cudaStreamCreateWithFlags(&st.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&st.done, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            release_all(s.get());
            return sfail(BANG_ECUDA, "bang_server_start: stream creation failed");
        }
        // one empty launch per stream allocates its work counter up front
        const Views dv = views(s->d_arena, s.get(), 1);
        const uint32_t one = 1, kL = cfg->k_max;
        cudaMemsetAsync(dv.q, 0, d * s->esz, st.stream);
        cudaMemcpyAsync(dv.k, &one, 4, cudaMemcpyHostToDevice, st.stream);
        cudaMemcpyAsync(dv.L, &kL, 4, cudaMemcpyHostToDevice, st.stream);
        bang_search_params p;
        std::memset(&p, 0, sizeof p);
        p.mode = cfg->mode;
        p.bloom_log2 = cfg->bloom_log2;
        p.early_codes = cfg->early_codes;
        int rc = bang_search_batched(ix, dv.q, 1, dv.k, dv.L, cfg->k_max, cfg->L_max, &p, dv.ids, dv.dist,
                                     st.stream);
        if (rc != BANG_OK || cudaStreamSynchronize(st.stream) != cudaSuccess) {
            std::string m = std::string("bang_server_start: warm-up search failed: ") + bang_last_error();
            release_all(s.get());
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
    if (batch_bytes(s, nq) > s->cap)
        return sfail(BANG_EINVAL, "bang_server_submit: the request needs more device memory than the "
                     "server's mem_bytes");
    auto r = std::make_shared<Request>();
    r->nq = nq;
    const auto *qb = static_cast<const unsigned char *>(queries);
    r->queries.assign(qb, qb + static_cast<size_t>(nq) * s->d * s->esz);
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
    release_all(s);
    delete s;
    return BANG_OK;
}

}  // extern "C"
