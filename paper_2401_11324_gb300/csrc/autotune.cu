// Autotuner for the search settings that do not change what the method
// computes, only how fast and how accurately this GPU runs it: the PQ table's
// precision and where it is built (§4.1: FP32, BF16 or 8-bit; per warp or on
// the tensor cores for the whole batch), the Bloom filter's size (§4.3, the
// paper's z), the persistent grid of the batched form, whether the graph rows
// are read packed, early code rows and the staged re-rank, and optionally
// the worklist size L that reaches a target recall.  Candidates are timed with
// CUDA events on the caller's stream and judged by recall@k against the
// caller's ground truth or, without one, against a high-accuracy FP32 search
// (2L, Bloom 2^18).  Decisions can be cached as JSON lines keyed by the GPU
// and the index's shape.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <mutex>
#include <sstream>
#include <string>
#include <unordered_set>
#include <vector>

#include "bang.h"
#include "bang_internal.h"

namespace {

struct Cfg {
    uint32_t mode, log2z, tsrc, grid_mult, L, layout;    // layout: BANG_GRAPH_PACKED | BANG_NEIGHBOR_CODES bits
    uint32_t depth = 1;                                   // prefetch depth
    uint32_t early = 0, rerank = 0;                       // early code rows, staged re-rank
};

struct Runner {
    bang_index *ix;
    const void *queries;
    uint32_t nq, k;
    bool batched;
    cudaStream_t st;
    uint32_t *d_ids = nullptr, *d_kq = nullptr, *d_Lq = nullptr;
    float *d_dist = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    std::vector<uint32_t> ids;

    int init(uint32_t L_max)
    {
        if (cudaMalloc(&d_ids, sizeof(uint32_t) * nq * k) != cudaSuccess ||
            cudaMalloc(&d_dist, sizeof(float) * nq * k) != cudaSuccess ||
            cudaMalloc(&d_kq, sizeof(uint32_t) * nq) != cudaSuccess ||
            cudaMalloc(&d_Lq, sizeof(uint32_t) * nq) != cudaSuccess) {
            cudaGetLastError();
            return BANG_ENOMEM;
        }
        if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
            cudaGetLastError();
            return BANG_ECUDA;
        }
        std::vector<uint32_t> kq(nq, k);
        if (cudaMemcpy(d_kq, kq.data(), sizeof(uint32_t) * nq, cudaMemcpyHostToDevice) != cudaSuccess)
            return BANG_ECUDA;
        (void)L_max;
        ids.resize(static_cast<size_t>(nq) * k);
        return BANG_OK;
    }
    ~Runner()
    {
        if (d_ids) cudaFree(d_ids);
        if (d_dist) cudaFree(d_dist);
        if (d_kq) cudaFree(d_kq);
        if (d_Lq) cudaFree(d_Lq);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    }
    int run(const Cfg &c)
    {
        bang_search_params p;
        std::memset(&p, 0, sizeof p);
        p.mode = c.mode;
        p.bloom_log2 = c.log2z;
        p.table_source = c.tsrc;
        p.grid_mult = c.grid_mult;
        p.prefetch_depth = c.depth;
        p.early_codes = c.early;
        p.rerank = c.rerank;
        if (!batched) return bang_search(ix, queries, nq, k, c.L, &p, d_ids, d_dist, st);
        std::vector<uint32_t> Lq(nq, c.L);
        if (cudaMemcpyAsync(d_Lq, Lq.data(), sizeof(uint32_t) * nq, cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return BANG_ECUDA;
        return bang_search_batched(ix, queries, nq, d_kq, d_Lq, k, c.L, &p, d_ids, d_dist, st);
    }
    // Mean milliseconds per batch over `reps` launches after one warm-up.
    int time(const Cfg &c, uint32_t reps, float *ms)
    {
        int rc = run(c);
        if (rc) return rc;
        float tot = 0.f;
        for (uint32_t r = 0; r < reps; ++r) {
            if (cudaEventRecord(e0, st) != cudaSuccess) return BANG_ECUDA;
            if ((rc = run(c))) return rc;
            float t = 0.f;
            if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&t, e0, e1) != cudaSuccess)
                return BANG_ECUDA;
            tot += t;
        }
        *ms = tot / static_cast<float>(reps ? reps : 1);
        return BANG_OK;
    }
    int fetch()
    {
        if (cudaStreamSynchronize(st) != cudaSuccess ||
            cudaMemcpy(ids.data(), d_ids, sizeof(uint32_t) * nq * k, cudaMemcpyDeviceToHost) != cudaSuccess)
            return BANG_ECUDA;
        return BANG_OK;
    }
};

// recall@k of `found` against `truth` (both nq*k; truth rows may hold
// 0xFFFFFFFF padding, which never counts).
float recall_at_k(const std::vector<uint32_t> &found, const uint32_t *truth, uint32_t nq, uint32_t k)
{
    uint64_t hit = 0, tot = 0;
    std::unordered_set<uint32_t> row;
    for (uint32_t q = 0; q < nq; ++q) {
        row.clear();
        for (uint32_t i = 0; i < k; ++i) row.insert(found[static_cast<size_t>(q) * k + i]);
        for (uint32_t i = 0; i < k; ++i) {
            const uint32_t t = truth[static_cast<size_t>(q) * k + i];
            if (t == 0xFFFFFFFFu) continue;
            ++tot;
            hit += row.count(t);
        }
    }
    return tot ? static_cast<float>(static_cast<double>(hit) / static_cast<double>(tot)) : 1.0f;
}

std::mutex g_cache_mu;

std::string cache_key(bang_index *ix, uint32_t nq, uint32_t k, uint32_t L, const bang_autotune_opts &o,
                      bool truth)
{
    uint64_t n = 0;
    uint32_t d = 0, M = 0, R = 0;
    int32_t dt = -1;
    bang_index_info(ix, &n, &d, &M, &R, &dt);
    int dev = bang::index_device(ix);
    cudaDeviceProp prop;
    std::memset(&prop, 0, sizeof prop);
    cudaGetDeviceProperties(&prop, dev);
    std::ostringstream s;
    s << "gpu=" << prop.name << "/sm" << prop.multiProcessorCount << "|n=" << n << "|d=" << d
      << "|M=" << M << "|R=" << R << "|dtype=" << dt << "|placement=" << bang::index_placement(ix)
      << "|nq=" << nq << "|k=" << k << "|L=" << L << "|target=" << o.target_recall
      << "|tol=" << o.recall_tolerance << "|modes=" << o.modes << "|bloom=" << o.bloom_min << "-"
      << o.bloom_max << "|tc=" << o.try_tensor_tables << "|batched=" << o.batched
      << "|packed=" << o.try_packed_graph << "|ncodes=" << o.try_neighbor_codes
      << "|depth=" << o.try_prefetch_depth << "|records=" << o.try_node_records
      << "|structure=" << o.try_structure << "|truth=" << (truth ? 1 : 0);
    std::string r = s.str();
    for (char &c : r)
        if (c == '"' || c == '\\' || c == '\n') c = '_';
    return r;
}

// Field `name` of a JSON line written by store(), as a number.
bool field(const std::string &line, const char *name, double *v)
{
    const std::string pat = std::string("\"") + name + "\": ";
    const size_t p = line.find(pat);
    if (p == std::string::npos) return false;
    return std::sscanf(line.c_str() + p + pat.size(), "%lf", v) == 1;
}

bool lookup(const char *path, const std::string &key, bang_autotune_result *out)
{
    std::lock_guard<std::mutex> lk(g_cache_mu);
    std::ifstream f(path);
    if (!f) return false;
    const std::string kpat = "{\"key\": \"" + key + "\",";
    std::string line, hit;
    while (std::getline(f, line))
        if (line.compare(0, kpat.size(), kpat) == 0) hit = line;    // the last entry wins
    if (hit.empty()) return false;
    double v[16];
    const char *names[16] = {"mode", "bloom_log2", "table_source", "grid_mult", "L", "ms", "recall",
                             "ref_ms", "ref_recall", "candidates", "graph_packed", "neighbor_codes",
                             "prefetch_depth", "node_records", "early_codes", "rerank"};
    for (int i = 0; i < 16; ++i)
        if (!field(hit, names[i], &v[i])) return false;
    out->mode = static_cast<uint32_t>(v[0]);
    out->bloom_log2 = static_cast<uint32_t>(v[1]);
    out->table_source = static_cast<uint32_t>(v[2]);
    out->grid_mult = static_cast<uint32_t>(v[3]);
    out->L = static_cast<uint32_t>(v[4]);
    out->ms = static_cast<float>(v[5]);
    out->recall = static_cast<float>(v[6]);
    out->ref_ms = static_cast<float>(v[7]);
    out->ref_recall = static_cast<float>(v[8]);
    out->candidates = static_cast<uint32_t>(v[9]);
    out->graph_packed = static_cast<uint32_t>(v[10]);
    out->neighbor_codes = static_cast<uint32_t>(v[11]);
    out->prefetch_depth = static_cast<uint32_t>(v[12]);
    out->node_records = static_cast<uint32_t>(v[13]);
    out->early_codes = static_cast<uint32_t>(v[14]);
    out->rerank = static_cast<uint32_t>(v[15]);
    out->from_cache = 1;
    return true;
}

void store(const char *path, const std::string &key, const bang_autotune_result &r)
{
    std::lock_guard<std::mutex> lk(g_cache_mu);
    std::ofstream f(path, std::ios::app);
    if (!f) return;
    char buf[512];
    std::snprintf(buf, sizeof buf,
                  "\"mode\": %u, \"bloom_log2\": %u, \"table_source\": %u, \"grid_mult\": %u, "
                  "\"L\": %u, \"ms\": %.6g, \"recall\": %.6g, \"ref_ms\": %.6g, \"ref_recall\": %.6g, "
                  "\"candidates\": %u, \"graph_packed\": %u, \"neighbor_codes\": %u, "
                  "\"prefetch_depth\": %u, \"node_records\": %u, \"early_codes\": %u, \"rerank\": %u}",
                  r.mode, r.bloom_log2, r.table_source, r.grid_mult, r.L, r.ms, r.recall, r.ref_ms,
                  r.ref_recall, r.candidates, r.graph_packed, r.neighbor_codes, r.prefetch_depth,
                  r.node_records, r.early_codes, r.rerank);
    f << "{\"key\": \"" << key << "\", " << buf << "\n";
}

int tfail(int code, const char *msg)
{
    bang::set_error(msg);
    return code;
}

}  // namespace

extern "C" int bang_autotune(bang_index *ix, const void *queries, uint32_t nq, uint32_t k, uint32_t L,
                             const uint32_t *truth, const bang_autotune_opts *opts,
                             bang_autotune_result *out, void *stream)
{
    if (!ix || !queries || !out) return tfail(BANG_EINVAL, "bang_autotune: NULL argument");
    if (nq == 0 || k == 0) return tfail(BANG_EINVAL, "bang_autotune: nq and k must be positive");
    bang_autotune_opts o;
    std::memset(&o, 0, sizeof o);
    if (opts) o = *opts;
    if (o.modes == 0) o.modes = (1u << BANG_MODE_PQ_F32) | (1u << BANG_MODE_PQ_BF16) | (1u << BANG_MODE_PQ_Q8);
    if (o.modes & ~0xFu) return tfail(BANG_EINVAL, "bang_autotune: unknown mode bit");
    if (o.bloom_min == 0) o.bloom_min = 13;
    if (o.bloom_max == 0) o.bloom_max = 17;
    if (o.bloom_min < 10 || o.bloom_max > 20 || o.bloom_min > o.bloom_max)
        return tfail(BANG_EINVAL, "bang_autotune: Bloom sizes must satisfy 10 <= min <= max <= 20");
    if (o.recall_tolerance <= 0.f) o.recall_tolerance = 0.005f;
    if (o.reps == 0) o.reps = 3;
    if (o.target_recall < 0.f || o.target_recall > 1.f)
        return tfail(BANG_EINVAL, "bang_autotune: target_recall outside 0..1");
    if (o.target_recall == 0.f && (L < k || L > 1024u))
        return tfail(BANG_EINVAL, "bang_autotune: need k <= L <= 1024 when no target recall is given");
    std::memset(out, 0, sizeof *out);

    const std::string key = cache_key(ix, nq, k, L, o, truth != nullptr);
    if (o.cache_path && lookup(o.cache_path, key, out)) return BANG_OK;

    // worklist sizes: the given L, or the sweep for the target recall
    std::vector<uint32_t> Ls;
    if (o.target_recall > 0.f) {
        for (uint32_t c : {16u, 24u, 32u, 48u, 64u, 80u, 96u, 112u, 128u, 160u, 192u, 224u, 256u, 288u, 320u,
                            384u, 512u, 768u, 1024u})
            if (c >= k && (L == 0 || c <= L)) Ls.push_back(c);
        if (Ls.empty()) return tfail(BANG_EINVAL, "bang_autotune: no worklist size between k and L");
    } else {
        Ls.push_back(L);
    }
    const uint32_t L_hi = Ls.back();

    Runner run{ix, queries, nq, k, o.batched != 0, static_cast<cudaStream_t>(stream)};
    int rc = run.init(L_hi);
    if (rc) return tfail(rc, "bang_autotune: scratch allocation failed");

    // accuracy reference: the caller's truth, or a wide FP32 search
    std::vector<uint32_t> pseudo;
    const uint32_t *ref_ids = truth;
    if (!ref_ids) {
        const uint32_t Lr = std::min(1024u, std::max(2u * L_hi, k));
        Runner wide{ix, queries, nq, k, false, static_cast<cudaStream_t>(stream)};
        if ((rc = wide.init(Lr))) return tfail(rc, "bang_autotune: scratch allocation failed");
        if ((rc = wide.run({BANG_MODE_PQ_F32, 18u, 0u, 0u, Lr, 0u})) || (rc = wide.fetch())) return rc;
        pseudo = wide.ids;
        ref_ids = pseudo.data();
    }

    // candidates
    // graph layouts to try: the caller's, plus packed rows and/or neighbour
    // codes when asked for (the latter only where the index allows it)
    const uint32_t place0 = bang::index_placement(ix);
    const uint32_t kLay = BANG_GRAPH_PACKED | BANG_NEIGHBOR_CODES;
    std::vector<uint32_t> layouts = {place0 & kLay};
    {
        uint64_t n_ = 0;
        uint32_t d_ = 0, M_ = 0, R_ = 0;
        int32_t dt_ = -1;
        bang_index_info(ix, &n_, &d_, &M_, &R_, &dt_);
        const bool nc_ok = R_ <= 64 && d_ <= 128 && M_ <= 32;
        for (uint32_t pk = 0; pk < 2; ++pk)
            for (uint32_t nc = 0; nc < 2; ++nc) {
                if ((pk && !o.try_packed_graph) || (nc && !(o.try_neighbor_codes && nc_ok))) continue;
                const uint32_t l = (pk ? BANG_GRAPH_PACKED : 0u) | (nc ? BANG_NEIGHBOR_CODES : 0u);
                if (std::find(layouts.begin(), layouts.end(), l) == layouts.end()) layouts.push_back(l);
            }
    }
    std::vector<Cfg> cands;
    for (uint32_t lay : layouts)
        for (uint32_t m = 0; m < 4; ++m) {
            if (!(o.modes & (1u << m))) continue;
            for (uint32_t z = o.bloom_min; z <= o.bloom_max; ++z) {
                std::vector<uint32_t> gms = {0u};
                if (o.batched) gms = {1u, 2u, 4u};
                for (uint32_t gm : gms) {
                    cands.push_back({m, z, 0u, gm, 0u, lay});
                    if (m == BANG_MODE_PQ_BF16 && o.try_tensor_tables) cands.push_back({m, z, 1u, gm, 0u, lay});
                }
            }
        }
    // the caller's placement, restored on every way out
    struct Restore {
        bang_index *ix;
        uint32_t flags;
        ~Restore() { if (bang::index_placement(ix) != flags) bang_set_placement(ix, flags); }
    } restore{ix, place0};
    uint32_t cur_lay = place0 & kLay;

    // the plain form at the default filter: the reference for the tolerance
    // (fixed L) and for the reported speed-up
    float ref_ms = 0.f, ref_acc = 0.f;
    {
        Cfg c{BANG_MODE_PQ_F32, 16u, 0u, o.batched ? 1u : 0u, Ls[0], cur_lay};
        if (o.target_recall > 0.f) {
            for (uint32_t Lc : Ls) {
                c.L = Lc;
                if ((rc = run.run(c)) || (rc = run.fetch())) return rc;
                ref_acc = recall_at_k(run.ids, ref_ids, nq, k);
                if (ref_acc >= o.target_recall) break;
            }
        } else {
            if ((rc = run.run(c)) || (rc = run.fetch())) return rc;
            ref_acc = recall_at_k(run.ids, ref_ids, nq, k);
        }
        if ((rc = run.time(c, o.reps, &ref_ms))) return rc;
    }

    bool found = false;
    uint32_t tried = 0;
    Cfg best_c{};
    for (Cfg c : cands) {
        if (c.layout != cur_lay) {
            if ((rc = bang_set_placement(ix, (place0 & ~kLay) | c.layout))) return rc;
            cur_lay = c.layout;
        }
        bool ok = false;
        float acc = 0.f;
        for (uint32_t Lc : Ls) {
            c.L = Lc;
            rc = run.run(c);
            if (rc == BANG_EINVAL) break;              // e.g. tensor-core tables unavailable here
            if (rc || (rc = run.fetch())) return rc;
            acc = recall_at_k(run.ids, ref_ids, nq, k);
            ok = o.target_recall > 0.f ? acc >= o.target_recall : acc >= ref_acc - o.recall_tolerance;
            if (ok || o.target_recall == 0.f) break;
        }
        if (rc == BANG_EINVAL) continue;
        ++tried;
        if (!ok) continue;
        float ms = 0.f;
        if ((rc = run.time(c, o.reps, &ms))) return rc;
        if (!found || ms < out->ms) {
            found = true;
            out->mode = c.mode;
            out->bloom_log2 = c.log2z;
            out->table_source = c.tsrc;
            out->grid_mult = c.grid_mult;
            out->L = c.L;
            out->ms = ms;
            out->recall = acc;
            out->graph_packed = (cur_lay & BANG_GRAPH_PACKED) ? 1u : 0u;
            out->neighbor_codes = (cur_lay & BANG_NEIGHBOR_CODES) ? 1u : 0u;
            out->prefetch_depth = 1;
            best_c = c;
        }
    }
    out->ref_ms = ref_ms;
    out->ref_recall = ref_acc;
    out->candidates = tried;
    if (!found) return tfail(BANG_EINVAL, "bang_autotune: no candidate reached the target recall");
    out->node_records = 0;
    if (best_c.layout != cur_lay) {
        if ((rc = bang_set_placement(ix, (place0 & ~kLay) | best_c.layout))) return rc;
        cur_lay = best_c.layout;
    }
    if (o.try_node_records && !(place0 & (BANG_GRAPH_IN_HBM | BANG_VECTORS_IN_HBM | BANG_NODE_RECORDS))) {
        // the winner with each node's row and vector side by side (same results)
        if ((rc = bang_set_placement(ix, (place0 & ~kLay) | best_c.layout | BANG_NODE_RECORDS))) return rc;
        float msr = 0.f;
        if ((rc = run.time(best_c, o.reps, &msr))) return rc;
        ++out->candidates;
        if (msr < out->ms) {
            out->ms = msr;
            out->node_records = 1;
        } else if ((rc = bang_set_placement(ix, (place0 & ~kLay) | best_c.layout))) {
            return rc;
        }
    }
    if (o.try_prefetch_depth) {       // the winner with the speculative request too (same results)
        Cfg c2 = best_c;
        c2.depth = 2;
        float ms2 = 0.f;
        if ((rc = run.time(c2, o.reps, &ms2))) return rc;
        ++out->candidates;
        if (ms2 < out->ms) {
            out->ms = ms2;
            out->prefetch_depth = 2;
            best_c = c2;
        }
    }
    if (o.try_structure && best_c.mode != BANG_MODE_EXACT) {
        // the winner with early code rows, then with the re-rank staged
        // (same results: each kept only if faster)
        Cfg c3 = best_c;
        c3.early = 1;
        float ms3 = 0.f;
        if ((rc = run.time(c3, o.reps, &ms3))) return rc;
        ++out->candidates;
        if (ms3 < out->ms) {
            out->ms = ms3;
            out->early_codes = 1;
            best_c = c3;
        }
        Cfg c4 = best_c;
        c4.rerank = 1;
        float ms4 = 0.f;
        if ((rc = run.time(c4, o.reps, &ms4))) return rc;
        ++out->candidates;
        if (ms4 < out->ms) {
            out->ms = ms4;
            out->rerank = 1;
        }
    }
    if (o.cache_path) store(o.cache_path, key, *out);
    return BANG_OK;
}
