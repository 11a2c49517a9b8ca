// GPU build of the overlapping-shard graph (§2.2: the paper's Vamana index
// is built by splitting the dataset into smaller overlapping clusters,
// building a directed subgraph on each with GreedySearch and RobustPrune, and
// merging the subgraphs' edges).  The steps, in the batched form whose
// results do not depend on thread scheduling:
//  1. each point joins the shards of its ell nearest centres (FP32 squared
//     distance, ascending dimension, each difference, product and sum
//     rounded; ties to the smaller centre);
//  2. a shard lists its members in ascending point id; its entry is the
//     member nearest its centre (ties to the smaller id); it inserts the
//     entry first, then the other members in ascending id;
//  3. two passes (pruning parameter 1, then alpha), each cutting every
//     shard's insertion order into batches (pass 1: 1, 1, 2, 4, ... up to
//     cap = max(1, floor(batch_frac * m)); pass 2: cap each); batch r of
//     every shard forms round r.  In a round, against the graph as it stood
//     at the round's start, each member runs GreedySearch from its shard's
//     entry (the search kernel in its exact-distance mode, worklist Lb, the
//     Bloom seen set, at most iter_cap expansions); its list becomes
//     RobustPrune(member, expanded U current list); then every node named by
//     a new list takes the members that named it (sorted union when it fits
//     in R, else RobustPrune of the union);
//  4. a point's final row is the union of its shard lists, as point ids,
//     sorted when it fits in R, else RobustPrune'd with alpha.
// Distances are the search kernel's exact distance rounded to FP32 (integer
// data exact; f32 as 32 partial sums of ascending dimensions, lane r owning
// the dimensions j with (j/4) mod 32 = r, fmaf, then an xor butterfly 16..1).
// Candidate lists are sorted by (distance, id), repeats and the owner
// removed, and cut to their 750 nearest (DiskANN's bound on the candidate
// pool; only reverse edges into hub nodes reach it).  RobustPrune: in that order a live candidate is kept (at most R)
// and removes every later candidate c with a^2 * d(kept, c) <= d(owner, c),
// a^2 and the product rounded to FP32.
//
// Layout: one device record per (point, shard) pair ("virtual node"): its
// row of R virtual ids, then its vector padded to 16 bytes, the record
// rounded to 32 bytes, so a GreedySearch expansion reads one contiguous
// record.  Prune work is one warp per list; for integer vectors of at most
// 128 bytes every lane holds its candidates' vectors in registers, so each
// kept neighbour costs one broadcast of its vector from shared memory and
// dp4a arithmetic per candidate (no per-pair memory traffic).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "bang.h"
#include "bang_internal.h"
#include "search_kernel.cuh"

namespace {

constexpr uint32_t kNo = 0xFFFFFFFFu;
constexpr int kW = 32;
constexpr int kKPL = 2;                  // candidates per lane per prune block (registers)
constexpr uint32_t kRegWords = 32;       // integer vectors of at most 128 bytes sit in registers
constexpr uint32_t kSmallC = 512;        // candidates of a list sorted by one warp in shared memory
constexpr uint32_t kCandCap = 750;       // RobustPrune looks at the nearest 750 candidates at most
constexpr uint32_t kKeySlots = 768;      // shared key slots: >= kSmallC and >= kCandCap
constexpr size_t kSmemMax = 227u * 1024u;
constexpr uint32_t kChunk = 1u << 20;    // searches per launch
constexpr int kScanT = 1024;

int sfail(int code, const std::string &m)
{
    bang::set_error(m);
    return code;
}

template <typename T> struct DBuf {
    T *p = nullptr;
    uint64_t n = 0;
    cudaError_t alloc(uint64_t count)
    {
        if (count <= n && p) return cudaSuccess;
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
        cudaError_t e = cudaMalloc(&p, sizeof(T) * (count ? count : 1));
        if (e == cudaSuccess) n = count;
        return e;
    }
    void release()
    {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
    ~DBuf() { release(); }
};

enum { kJobFwd = 0, kJobRev = 1, kJobMerge = 2 };

struct LArgs {
    const uint32_t *rec;     // virtual-node records
    uint32_t *recw;
    uint32_t rec_words, vec_off, vwords;   // record words, vector offset (words), vector words
    int dtype;
    uint32_t d, R, ell;
    float a2;
    int always_prune;        // forward lists are always pruned (the list is rebuilt)
    int kind;                // kJob*
    uint32_t njobs;
    // forward jobs: members[b], its expansions trace[b * tcap .. + iters[b]), out staging[b]
    const uint32_t *members;
    const uint32_t *trace, *iters;
    uint32_t tcap;
    uint32_t *staging;
    // reverse jobs: target touched[t], sources in_src[in_off[t] .. + in_cnt[t])
    const uint32_t *touched;
    const uint64_t *in_off;
    const uint32_t *in_cnt, *in_src;
    // merge jobs: points p0 + j; their virtual nodes vid[p * ell + t]; vpt maps back;
    // vfirst[p] = the first virtual node of p (where its vector is read)
    uint64_t p0;
    const uint32_t *vid, *vpt;
    uint32_t *out_rows;      // merge output, njobs rows of R
    // lists longer than kSmallC, handed to big_list_kernel
    uint32_t *defer, *ndefer;
};

__device__ __forceinline__ const uint32_t *vec_ptr(const LArgs &a, uint32_t v)
{
    return a.rec + static_cast<uint64_t>(v) * a.rec_words + a.vec_off;
}
// The vector of a candidate: virtual id (forward, reverse) or point id (merge).
__device__ __forceinline__ const uint32_t *cand_vec(const LArgs &a, uint32_t id)
{
    return a.kind == kJobMerge ? vec_ptr(a, a.vid[static_cast<uint64_t>(id) * a.ell]) : vec_ptr(a, id);
}

// Integer squared distance over `nw` words (padding bytes are zero on both sides).
template <int DT>
__device__ __forceinline__ uint32_t idist(const uint32_t *x, const uint32_t *y, uint32_t nw)
{
    uint32_t acc = 0;
    for (uint32_t w = 0; w < nw; ++w) {
        const uint32_t t = DT == 1 ? __vabsdiffs4(x[w], y[w]) : __vabsdiffu4(x[w], y[w]);
        acc = __dp4a(t, t, acc);
    }
    return acc;
}

// The same with x held in registers (every index static).
template <int DT>
__device__ __forceinline__ uint32_t idist_reg(const uint32_t (&x)[kRegWords], const uint32_t *y, uint32_t nw)
{
    uint32_t acc = 0;
#pragma unroll
    for (uint32_t w = 0; w < kRegWords; ++w) {
        if (w < nw) {
            const uint32_t t = DT == 1 ? __vabsdiffs4(x[w], y[w]) : __vabsdiffu4(x[w], y[w]);
            acc = __dp4a(t, t, acc);
        }
    }
    return acc;
}

// FP32 exact distance in the search kernel's order (see the file comment).
__device__ float fdist(const float *x, const float *y, uint32_t d)
{
    float p[32];
#pragma unroll
    for (int r = 0; r < 32; ++r) {
        float acc = 0.0f;
        for (uint32_t j0 = 4u * r; j0 < d; j0 += 128u)
            for (uint32_t t = 0; t < 4u && j0 + t < d; ++t) {
                const float df = __fsub_rn(x[j0 + t], y[j0 + t]);
                acc = __fmaf_rn(df, df, acc);
            }
        p[r] = acc;
    }
#pragma unroll
    for (int h = 16; h >= 1; h >>= 1) {
        float nx[32];
#pragma unroll
        for (int r = 0; r < 32; ++r) nx[r] = __fadd_rn(p[r], p[r ^ h]);
#pragma unroll
        for (int r = 0; r < 32; ++r) p[r] = nx[r];
    }
    return p[0];
}

template <int DT>
__device__ __forceinline__ float vdist(const LArgs &a, const uint32_t *x, const uint32_t *y)
{
    if (DT == 2) return fdist(reinterpret_cast<const float *>(x), reinterpret_cast<const float *>(y), a.d);
    return __uint2float_rn(idist<DT>(x, y, a.vwords));
}

__device__ __forceinline__ uint64_t mkkey(float dist, uint32_t id)
{
    return (static_cast<uint64_t>(__float_as_uint(dist)) << 32) | id;
}
__device__ __forceinline__ uint32_t kid(uint64_t k) { return static_cast<uint32_t>(k); }
__device__ __forceinline__ float kdist(uint64_t k) { return __uint_as_float(static_cast<uint32_t>(k >> 32)); }

// Candidate ids of a job (the owner excluded later): forward = its
// expansions then its current row; reverse = its current row then the
// members that named it; merge = its shards' rows as point ids.  Writes
// ids[i] for i < returned count when the count is at most cap.
__device__ __forceinline__ uint32_t job_candidates(const LArgs &a, uint32_t job, uint32_t cap, uint32_t *ids,
                                                   uint32_t &owner, int tid, int nthreads)
{
    uint32_t C;
    if (a.kind == kJobFwd) {
        owner = a.members[job];
        const uint32_t ni = min(a.iters[job], a.tcap);
        C = ni + a.R;
        if (C <= cap) {
            for (uint32_t i = tid; i < ni; i += nthreads) ids[i] = a.trace[static_cast<uint64_t>(job) * a.tcap + i];
            for (uint32_t i = tid; i < a.R; i += nthreads)
                ids[ni + i] = a.rec[static_cast<uint64_t>(owner) * a.rec_words + i];
        }
    } else if (a.kind == kJobRev) {
        owner = a.touched[job];
        const uint32_t ni = a.in_cnt[job];
        C = ni + a.R;
        if (C <= cap) {
            for (uint32_t i = tid; i < a.R; i += nthreads) ids[i] = a.rec[static_cast<uint64_t>(owner) * a.rec_words + i];
            for (uint32_t i = tid; i < ni; i += nthreads) ids[a.R + i] = a.in_src[a.in_off[job] + i];
        }
    } else {
        owner = static_cast<uint32_t>(a.p0 + job);
        C = a.ell * a.R;
        if (C <= cap) {
            for (uint32_t i = tid; i < C; i += nthreads) {
                const uint32_t v = a.vid[static_cast<uint64_t>(owner) * a.ell + i / a.R];
                const uint32_t q = a.rec[static_cast<uint64_t>(v) * a.rec_words + i % a.R];
                ids[i] = q == kNo ? kNo : a.vpt[q];
            }
        }
    }
    return C;
}

__device__ __forceinline__ const uint32_t *owner_vec(const LArgs &a, uint32_t owner)
{
    return a.kind == kJobMerge ? cand_vec(a, owner) : vec_ptr(a, owner);
}

__device__ __forceinline__ uint32_t *job_out(const LArgs &a, uint32_t job, uint32_t owner)
{
    return a.kind == kJobFwd ? a.staging + static_cast<uint64_t>(job) * a.R
         : a.kind == kJobRev ? a.recw + static_cast<uint64_t>(owner) * a.rec_words
                             : a.out_rows + static_cast<uint64_t>(job) * a.R;
}

// Compact C sorted keys (from `src`, shared or global) into dst without
// repeats or invalid keys, keeping at most kCandCap; returns the count.  The
// key before each 32-key chunk is carried in a register, since the
// compaction may overwrite its slot when src == dst.  One warp.
__device__ __forceinline__ uint32_t dedupe_keys(const uint64_t *src, uint32_t C, uint64_t *dst, int lane)
{
    uint32_t u = 0;
    uint64_t last = ~0ull;                 // id part 0xFFFFFFFF: no valid id
    for (uint32_t c0 = 0; c0 < C && u < kCandCap; c0 += kW) {
        const uint32_t i = c0 + lane;
        const uint64_t x = i < C ? src[i] : ~0ull;
        uint64_t prev = __shfl_up_sync(0xFFFFFFFFu, x, 1);
        if (lane == 0) prev = last;
        last = __shfl_sync(0xFFFFFFFFu, x, kW - 1);
        const bool keep = x != ~0ull && kid(prev) != kid(x);
        __syncwarp();
        const uint32_t bal = __ballot_sync(0xFFFFFFFFu, keep);
        const uint32_t pos = u + __popc(bal & ((1u << lane) - 1u));
        if (keep && pos < kCandCap) dst[pos] = x;
        u = min(u + __popc(bal), kCandCap);
        __syncwarp();
    }
    return u;
}

// The list of `owner` from u sorted unique keys (shared memory): the keys
// themselves when they fit in R and the job does not always prune, else
// RobustPrune over them, 32 * kKPL candidates at a time.  One warp.
template <int DT>
__device__ void finish_list(const LArgs &a, const uint64_t *keys, uint32_t u, const uint32_t *ovec,
                            uint32_t *kvec, uint32_t *kept, uint32_t *out, int lane)
{
    const bool regs = DT != 2 && a.vwords <= kRegWords;
    if (u <= a.R && !a.always_prune) {
        for (uint32_t i = lane; i < a.R; i += kW) out[i] = i < u ? kid(keys[i]) : kNo;
        __syncwarp();
        return;
    }
    uint32_t nout = 0;
    for (uint32_t b0 = 0; b0 < u && nout < a.R; b0 += kW * kKPL) {
        uint32_t cid[kKPL];
        float dp[kKPL];
        bool alive[kKPL];
        uint32_t cv[kKPL][kRegWords];
#pragma unroll
        for (int s = 0; s < kKPL; ++s) {
            const uint32_t i = b0 + s * kW + lane;
            alive[s] = i < u;
            cid[s] = alive[s] ? kid(keys[i]) : kNo;
            dp[s] = alive[s] ? kdist(keys[i]) : 0.0f;
            if (regs) {
                const uint32_t *src = alive[s] ? cand_vec(a, cid[s]) : ovec;
#pragma unroll
                for (uint32_t w = 0; w < kRegWords; ++w) cv[s][w] = w < a.vwords ? src[w] : 0u;
            }
        }
        // kept neighbours of earlier blocks
        for (uint32_t t = 0; t < nout; ++t) {
            const uint32_t *kv = kvec + t * a.vwords;
#pragma unroll
            for (int s = 0; s < kKPL; ++s) {
                if (!alive[s]) continue;
                const float dd = regs ? __uint2float_rn(idist_reg<DT>(cv[s], kv, a.vwords))
                                      : vdist<DT>(a, kv, cand_vec(a, cid[s]));
                if (__fmul_rn(a.a2, dd) <= dp[s]) alive[s] = false;
            }
        }
        // walk this block in order
        for (uint32_t pos = 0; pos < kW * kKPL && b0 + pos < u && nout < a.R; ++pos) {
            const int s = static_cast<int>(pos / kW), l = static_cast<int>(pos % kW);
            bool mine = false;
#pragma unroll
            for (int t = 0; t < kKPL; ++t) if (t == s) mine = alive[t];
            if (!__shfl_sync(0xFFFFFFFFu, mine ? 1 : 0, l)) continue;
            uint32_t *kv = kvec + nout * a.vwords;
            if (lane == l) {
#pragma unroll
                for (int t = 0; t < kKPL; ++t) {
                    if (t != s) continue;
                    kept[nout] = cid[t];
                    alive[t] = false;
                    if (regs) {
#pragma unroll
                        for (uint32_t w = 0; w < kRegWords; ++w) if (w < a.vwords) kv[w] = cv[t][w];
                    }
                }
            }
            if (!regs) {
                const uint32_t kid_ = __shfl_sync(0xFFFFFFFFu, lane == l ? kept[nout] : 0u, l);
                const uint32_t *src = cand_vec(a, kid_);
                for (uint32_t w = lane; w < a.vwords; w += kW) kv[w] = src[w];
            }
            __syncwarp();
#pragma unroll
            for (int t = 0; t < kKPL; ++t) {
                if (!alive[t]) continue;
                const float dd = regs ? __uint2float_rn(idist_reg<DT>(cv[t], kv, a.vwords))
                                      : vdist<DT>(a, kv, cand_vec(a, cid[t]));
                if (__fmul_rn(a.a2, dd) <= dp[t]) alive[t] = false;
            }
            ++nout;
        }
        __syncwarp();
    }
    __syncwarp();
    for (uint32_t i = lane; i < a.R; i += kW) out[i] = i < nout ? kept[i] : kNo;
    __syncwarp();
}

// Shared memory of a list (both kernels): kKeySlots keys, kSmallC ids, the
// owner's vector, the kept vectors (R) and ids.
struct ListSmem {
    uint64_t *keys;
    uint32_t *ids, *ovec, *kvec, *kept;
    __device__ ListSmem(unsigned char *sm, const LArgs &a)
    {
        keys = reinterpret_cast<uint64_t *>(sm);
        ids = reinterpret_cast<uint32_t *>(keys + kKeySlots);
        ovec = ids + kSmallC;
        kvec = ovec + a.vwords;
        kept = kvec + a.R * a.vwords;
    }
};

// One warp per list of at most kSmallC candidates; longer lists are listed
// in a.defer for big_list_kernel.
template <int DT>
__global__ void __launch_bounds__(32) list_kernel(const LArgs a)
{
    extern __shared__ __align__(16) unsigned char sm[];
    const int lane = threadIdx.x;
    const ListSmem m(sm, a);
    for (uint32_t job = blockIdx.x; job < a.njobs; job += gridDim.x) {
        uint32_t owner = 0;
        const uint32_t C = job_candidates(a, job, kSmallC, m.ids, owner, lane, kW);
        if (C > kSmallC) {
            if (lane == 0) a.defer[atomicAdd(a.ndefer, 1u)] = job;
            __syncwarp();
            continue;
        }
        const uint32_t *ovp = owner_vec(a, owner);
        for (uint32_t w = lane; w < a.vwords; w += kW) m.ovec[w] = ovp[w];
        __syncwarp();
        // keys (distance to the owner, id); invalid entries sort last
        uint32_t P = 32;
        while (P < C) P <<= 1;
        for (uint32_t i = lane; i < P; i += kW) {
            uint64_t k = ~0ull;
            if (i < C) {
                const uint32_t id = m.ids[i];
                if (id != kNo && id != owner) k = mkkey(vdist<DT>(a, m.ovec, cand_vec(a, id)), id);
            }
            m.keys[i] = k;
        }
        __syncwarp();
        for (uint32_t k = 2; k <= P; k <<= 1)                    // bitonic sort, ascending
            for (uint32_t j = k >> 1; j > 0; j >>= 1) {
                for (uint32_t i = lane; i < P; i += kW) {
                    const uint32_t l = i ^ j;
                    if (l > i) {
                        const uint64_t x = m.keys[i], y = m.keys[l];
                        const bool up = (i & k) == 0;
                        if ((x > y) == up) { m.keys[i] = y; m.keys[l] = x; }
                    }
                }
                __syncwarp();
            }
        const uint32_t u = dedupe_keys(m.keys, C, m.keys, lane);
        finish_list<DT>(a, m.keys, u, m.ovec, m.kvec, m.kept, job_out(a, job, owner), lane);
    }
}

// Lists of more than kSmallC candidates (reverse edges of hub nodes): one
// 1024-thread CTA per list; the keys are computed and sorted (bitonic) in a
// global-memory region of the next power of two above the count, then warp 0
// keeps the kCandCap nearest unique ones and finishes the list.
template <int DT>
__global__ void __launch_bounds__(1024) big_list_kernel(const LArgs a, const uint32_t *jobs, uint32_t njobs,
                                                        const uint64_t *region_off, uint64_t *region)
{
    extern __shared__ __align__(16) unsigned char sm[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const ListSmem m(sm, a);
    for (uint32_t b = blockIdx.x; b < njobs; b += gridDim.x) {
        const uint32_t job = jobs[b];
        uint64_t *keys = region + region_off[b];
        uint32_t owner = 0;
        const uint32_t C = job_candidates(a, job, 0u, nullptr, owner, tid, blockDim.x);
        uint32_t P = 32;
        while (P < C) P <<= 1;
        const uint32_t *ovp = owner_vec(a, owner);
        for (uint32_t w = tid; w < a.vwords; w += blockDim.x) m.ovec[w] = ovp[w];
        __syncthreads();
        for (uint32_t i = tid; i < P; i += blockDim.x) {
            uint64_t k = ~0ull;
            if (i < C) {
                uint32_t id;
                if (a.kind == kJobRev)
                    id = i < a.R ? a.rec[static_cast<uint64_t>(owner) * a.rec_words + i]
                                 : a.in_src[a.in_off[job] + (i - a.R)];
                else
                    id = kNo;                 // only reverse lists exceed kSmallC
                if (id != kNo && id != owner) k = mkkey(vdist<DT>(a, m.ovec, cand_vec(a, id)), id);
            }
            keys[i] = k;
        }
        __syncthreads();
        for (uint32_t k = 2; k <= P; k <<= 1)
            for (uint32_t j = k >> 1; j > 0; j >>= 1) {
                for (uint32_t i = tid; i < P; i += blockDim.x) {
                    const uint32_t l = i ^ j;
                    if (l > i) {
                        const uint64_t x = keys[i], y = keys[l];
                        const bool up = (i & k) == 0;
                        if ((x > y) == up) { keys[i] = y; keys[l] = x; }
                    }
                }
                __syncthreads();
            }
        if (warp == 0) {
            const uint32_t u = dedupe_keys(keys, C, m.keys, lane);
            finish_list<DT>(a, m.keys, u, m.ovec, m.kvec, m.kept, job_out(a, job, owner), lane);
        }
        __syncthreads();
    }
}

// Region sizes of the big lists: the next power of two above each count.
__global__ void big_regions(const LArgs a, const uint32_t *jobs, uint32_t njobs, uint64_t *off,
                            unsigned long long *total)
{
    const uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= njobs) return;
    const uint32_t C = a.R + a.in_cnt[jobs[b]];
    uint32_t P = 32;
    while (P < C) P <<= 1;
    off[b] = atomicAdd(total, static_cast<unsigned long long>(P));
}

// ---- assignment: the ell nearest centres of every point; the shard entries
// as the smallest (distance, point id) key per shard
template <int DT>
__global__ void assign_kernel(const void *X, uint64_t n, uint32_t d, const float *centres, uint32_t S,
                              uint32_t ell, uint32_t *sh, float *shd)
{
    using E = typename bang::Elem<DT>::T;
    const uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const E *x = static_cast<const E *>(X) + i * d;
    float bd[4];
    uint32_t bg[4];
    for (uint32_t t = 0; t < ell; ++t) { bd[t] = __uint_as_float(0x7F800000u); bg[t] = kNo; }
    for (uint32_t g = 0; g < S; ++g) {
        const float *c = centres + static_cast<uint64_t>(g) * d;
        float acc = 0.0f;
        for (uint32_t j = 0; j < d; ++j) {
            const float t = __fsub_rn(static_cast<float>(x[j]), __ldg(c + j));
            acc = __fadd_rn(acc, __fmul_rn(t, t));
        }
        // insert (acc, g) into the ell smallest, ties to the smaller g (g ascends)
        if (bg[ell - 1] != kNo && !(acc < bd[ell - 1])) continue;
        uint32_t t = ell - 1;
        while (t > 0 && (bg[t - 1] == kNo || acc < bd[t - 1])) {
            bd[t] = bd[t - 1];
            bg[t] = bg[t - 1];
            --t;
        }
        bd[t] = acc;
        bg[t] = g;
    }
    for (uint32_t t = 0; t < ell; ++t) {
        sh[i * ell + t] = bg[t];
        shd[i * ell + t] = bd[t];
    }
}

__global__ void entry_kernel(const uint32_t *sh, const float *shd, uint64_t nv, uint32_t ell,
                             unsigned long long *ekey)
{
    const uint64_t k = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (k >= nv) return;
    // key (distance bits, point id): the member nearest the centre, ties to the smaller id
    atomicMin(ekey + sh[k], (static_cast<unsigned long long>(__float_as_uint(shd[k])) << 32) | (k / ell));
}

// ---- records: rows empty, vectors copied from the points
__global__ void records_init(uint32_t *rec, uint64_t nv, uint32_t rec_words, uint32_t R, uint32_t vec_off,
                             const unsigned char *X, uint32_t row_bytes, const uint32_t *vpt)
{
    const uint64_t k = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (k >= nv * rec_words) return;
    const uint64_t v = k / rec_words;
    const uint32_t w = static_cast<uint32_t>(k % rec_words);
    uint32_t val = 0;
    if (w < R) {
        val = kNo;
    } else if (w >= vec_off) {
        const uint32_t b0 = (w - vec_off) * 4u;
        const unsigned char *src = X + static_cast<uint64_t>(vpt[v]) * row_bytes;
        for (uint32_t t = 0; t < 4; ++t)
            if (b0 + t < row_bytes) val |= static_cast<uint32_t>(src[b0 + t]) << (8 * t);
    }
    rec[k] = val;
}

// ---- a round's searches: query vectors (rows of row_bytes, the layout the
// search kernel reads) and entries of the members
__global__ void gather_queries(const uint32_t *members, uint32_t cnt, const uint32_t *rec, uint32_t rec_words,
                               uint32_t vec_off, uint32_t row_bytes, const uint64_t *gstart, uint32_t S,
                               const uint32_t *ventry, unsigned char *qbuf, uint32_t *ebuf)
{
    const uint64_t k = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (k >= static_cast<uint64_t>(cnt) * row_bytes) return;
    const uint32_t b = static_cast<uint32_t>(k / row_bytes), t = static_cast<uint32_t>(k % row_bytes);
    const uint32_t v = members[b];
    const unsigned char *src = reinterpret_cast<const unsigned char *>(rec + static_cast<uint64_t>(v) * rec_words + vec_off);
    qbuf[k] = src[t];
    if (t == 0) {
        uint32_t lo = 0, hi = S;             // shard of v: gstart[lo] <= v < gstart[lo + 1]
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (gstart[mid] <= v) lo = mid; else hi = mid;
        }
        ebuf[b] = ventry[lo];
    }
}

__global__ void commit_rows(const uint32_t *members, uint32_t cnt, const uint32_t *staging, uint32_t R,
                            uint32_t *rec, uint32_t rec_words)
{
    const uint64_t k = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (k >= static_cast<uint64_t>(cnt) * R) return;
    rec[static_cast<uint64_t>(members[k / R]) * rec_words + k % R] = staging[k];
}

// ---- reverse edges: count per target (first count lists the target), scan, place
__global__ void rev_count(const uint32_t *staging, uint64_t nrows, uint32_t R, uint32_t *cnt,
                          uint32_t *tpos, uint32_t *touched, unsigned int *ntouched)
{
    const uint64_t k = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (k >= nrows * R) return;
    const uint32_t c = staging[k];
    if (c == kNo) return;
    if (atomicAdd(cnt + c, 1u) == 0u) {
        const uint32_t t = atomicAdd(ntouched, 1u);
        touched[t] = c;
        tpos[c] = t;
    }
}

__global__ void rev_counts_of_touched(const uint32_t *touched, uint32_t nt, const uint32_t *cnt, uint32_t *tc)
{
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < nt) tc[t] = cnt[touched[t]];
}

__global__ void rev_place(const uint32_t *staging, const uint32_t *members, uint64_t nrows, uint32_t R,
                          const uint32_t *tpos, const uint64_t *toff, uint32_t *fill, uint32_t *in_src)
{
    const uint64_t k = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (k >= nrows * R) return;
    const uint32_t c = staging[k];
    if (c == kNo) return;
    const uint32_t t = tpos[c];
    in_src[toff[t] + atomicAdd(fill + t, 1u)] = members[k / R];
}

__global__ void rev_reset(const uint32_t *touched, uint32_t nt, uint32_t *cnt)
{
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < nt) cnt[touched[t]] = 0u;
}

// ---- exclusive scan of n 32-bit counts into 64-bit offsets
__global__ void scan_block_sums(const uint32_t *in, uint64_t n, uint64_t *bsum)
{
    __shared__ uint64_t s[kScanT];
    const uint64_t i = static_cast<uint64_t>(blockIdx.x) * kScanT + threadIdx.x;
    s[threadIdx.x] = i < n ? in[i] : 0u;
    __syncthreads();
    for (int h = kScanT / 2; h > 0; h >>= 1) {
        if (static_cast<int>(threadIdx.x) < h) s[threadIdx.x] += s[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) bsum[blockIdx.x] = s[0];
}

__global__ void scan_sums_exclusive(uint64_t *bsum, uint32_t nb)
{
    __shared__ uint64_t s[kScanT];
    uint64_t run = 0;
    for (uint32_t b0 = 0; b0 < nb; b0 += kScanT) {
        const uint32_t i = b0 + threadIdx.x;
        const uint64_t v = i < nb ? bsum[i] : 0;
        s[threadIdx.x] = v;
        __syncthreads();
        for (int h = 1; h < kScanT; h <<= 1) {
            const uint64_t add = static_cast<int>(threadIdx.x) >= h ? s[threadIdx.x - h] : 0;
            __syncthreads();
            s[threadIdx.x] += add;
            __syncthreads();
        }
        if (i < nb) bsum[i] = run + s[threadIdx.x] - v;
        run += s[kScanT - 1];
        __syncthreads();
    }
}

__global__ void scan_apply(const uint32_t *in, uint64_t n, const uint64_t *bsum, uint64_t *out)
{
    __shared__ uint64_t s[kScanT];
    const uint64_t i = static_cast<uint64_t>(blockIdx.x) * kScanT + threadIdx.x;
    const uint64_t v = i < n ? in[i] : 0u;
    s[threadIdx.x] = v;
    __syncthreads();
    for (int h = 1; h < kScanT; h <<= 1) {
        const uint64_t add = static_cast<int>(threadIdx.x) >= h ? s[threadIdx.x - h] : 0;
        __syncthreads();
        s[threadIdx.x] += add;
        __syncthreads();
    }
    if (i < n) out[i] = bsum[blockIdx.x] + s[threadIdx.x] - v;
}

uint32_t blocks(uint64_t work, uint32_t per) { return static_cast<uint32_t>((work + per - 1) / per); }

}  // namespace

#define SG_TRY(x)                                                                          \
    do {                                                                                   \
        cudaError_t e_ = (x);                                                              \
        if (e_ != cudaSuccess) {                                                           \
            cudaGetLastError();                                                            \
            return sfail(e_ == cudaErrorMemoryAllocation ? BANG_ENOMEM : BANG_ECUDA,       \
                         std::string("bang_build_shard_graph: ") + #x + ": " +             \
                             cudaGetErrorString(e_));                                      \
        }                                                                                  \
    } while (0)

namespace {

// Exclusive scan of n counts (device) into out (device, n entries).
cudaError_t scan_counts(const uint32_t *in, uint64_t n, uint64_t *out, DBuf<uint64_t> &bsum, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    const uint32_t nb = blocks(n, kScanT);
    cudaError_t e = bsum.alloc(nb);
    if (e != cudaSuccess) return e;
    scan_block_sums<<<nb, kScanT, 0, st>>>(in, n, bsum.p);
    scan_sums_exclusive<<<1, kScanT, 0, st>>>(bsum.p, nb);
    scan_apply<<<nb, kScanT, 0, st>>>(in, n, bsum.p, out);
    return cudaGetLastError();
}

size_t list_smem(uint32_t vwords, uint32_t R)
{
    return static_cast<size_t>(kKeySlots) * 8u + static_cast<size_t>(kSmallC) * 4u +
           4u * (vwords + static_cast<size_t>(R) * vwords + R) + 16u;
}

template <int DT> cudaError_t launch_small(const LArgs &a, size_t smem, uint32_t grid, cudaStream_t st)
{
    cudaError_t e = cudaFuncSetAttribute(list_kernel<DT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(kSmemMax));
    if (e != cudaSuccess) return e;
    list_kernel<DT><<<grid, 32, smem, st>>>(a);
    return cudaGetLastError();
}

template <int DT>
cudaError_t launch_big(const LArgs &a, const uint32_t *jobs, uint32_t nd, const uint64_t *off, uint64_t *region,
                       size_t smem, cudaStream_t st)
{
    cudaError_t e = cudaFuncSetAttribute(big_list_kernel<DT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(kSmemMax));
    if (e != cudaSuccess) return e;
    big_list_kernel<DT><<<std::min<uint32_t>(nd, 1024u), 1024, smem, st>>>(a, jobs, nd, off, region);
    return cudaGetLastError();
}

struct BigScratch {
    DBuf<uint32_t> defer, ndefer;
    DBuf<uint64_t> off, region;
    DBuf<unsigned long long> total;
};

// Every list of the launch: one warp per list of at most kSmallC candidates,
// then one CTA per longer list.
cudaError_t run_lists(LArgs a, BigScratch &bs, cudaStream_t st)
{
    if (a.njobs == 0) return cudaSuccess;
    cudaError_t e;
    if ((e = bs.defer.alloc(a.njobs)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(bs.ndefer.p, 0, 4, st)) != cudaSuccess) return e;
    a.defer = bs.defer.p;
    a.ndefer = bs.ndefer.p;
    const size_t smem = list_smem(a.vwords, a.R);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const uint32_t grid = std::min<uint32_t>(a.njobs, static_cast<uint32_t>(sms) * 64u);
    e = a.dtype == 0 ? launch_small<0>(a, smem, grid, st)
      : a.dtype == 1 ? launch_small<1>(a, smem, grid, st) : launch_small<2>(a, smem, grid, st);
    if (e != cudaSuccess) return e;
    uint32_t nd = 0;
    if ((e = cudaMemcpyAsync(&nd, bs.ndefer.p, 4, cudaMemcpyDeviceToHost, st)) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
    if (nd == 0) return cudaSuccess;
    if ((e = bs.off.alloc(nd)) != cudaSuccess) return e;
    if ((e = bs.total.alloc(1)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(bs.total.p, 0, 8, st)) != cudaSuccess) return e;
    big_regions<<<blocks(nd, 256), 256, 0, st>>>(a, bs.defer.p, nd, bs.off.p, bs.total.p);
    unsigned long long total = 0;
    if ((e = cudaMemcpyAsync(&total, bs.total.p, 8, cudaMemcpyDeviceToHost, st)) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
    if ((e = bs.region.alloc(total)) != cudaSuccess) return e;
    return a.dtype == 0 ? launch_big<0>(a, bs.defer.p, nd, bs.off.p, bs.region.p, smem, st)
         : a.dtype == 1 ? launch_big<1>(a, bs.defer.p, nd, bs.off.p, bs.region.p, smem, st)
                        : launch_big<2>(a, bs.defer.p, nd, bs.off.p, bs.region.p, smem, st);
}

}  // namespace

extern "C" int bang_build_shard_graph(int device, const void *base, bang_dtype dtype, uint64_t n, uint32_t d,
                                      const float *centres, uint32_t S, uint32_t ell, uint32_t R, uint32_t Lb,
                                      float alpha, float batch_frac, uint32_t log2z, uint32_t iter_cap,
                                      uint32_t *adj, uint32_t *shard_of, void *stream)
{
    if (!base || !centres || !adj) return sfail(BANG_EINVAL, "bang_build_shard_graph: NULL argument");
    if (dtype != BANG_U8 && dtype != BANG_I8 && dtype != BANG_F32)
        return sfail(BANG_EINVAL, "bang_build_shard_graph: unknown dtype");
    if (n == 0 || d == 0 || d > static_cast<uint32_t>(bang::kMaxD))
        return sfail(BANG_EINVAL, "bang_build_shard_graph: need n > 0 and 1 <= d <= 512");
    if (S == 0 || ell == 0 || ell > 4 || ell > S)
        return sfail(BANG_EINVAL, "bang_build_shard_graph: need S >= 1 and 1 <= ell <= min(4, S)");
    if (n * ell >= 0x7FFFFFFFull)
        return sfail(BANG_EINVAL, "bang_build_shard_graph: n * ell must stay below 2^31 - 1");
    if (R == 0 || R > 128 || R % 4 != 0 || ell * R > kSmallC)
        return sfail(BANG_EINVAL, "bang_build_shard_graph: R must be a multiple of 4 in 4..128 with ell * R <= 512");
    if (Lb == 0 || Lb > static_cast<uint32_t>(bang::kMaxL))
        return sfail(BANG_EINVAL, "bang_build_shard_graph: Lb outside 1..1024");
    if (log2z < 10 || log2z > 20) return sfail(BANG_EINVAL, "bang_build_shard_graph: log2z outside 10..20");
    if (iter_cap == 0) iter_cap = 2 * Lb + 64;
    if (iter_cap + R > kSmallC)
        return sfail(BANG_EINVAL, "bang_build_shard_graph: iter_cap + R must be at most 512");
    {
        const uint32_t vw = ((d * (dtype == BANG_F32 ? 4u : 1u) + 15u) & ~15u) / 4u;
        if (list_smem(vw, R) > kSmemMax)
            return sfail(BANG_EINVAL, "bang_build_shard_graph: R kept vectors of d dimensions exceed shared memory");
    }
    if (!(alpha >= 1.0f) || !(batch_frac > 0.0f) || !(batch_frac <= 1.0f))
        return sfail(BANG_EINVAL, "bang_build_shard_graph: need alpha >= 1 and 0 < batch_frac <= 1");
    if (bang::pointer_kind(base, device) == 2 || bang::pointer_kind(adj, device) == 2)
        return sfail(BANG_EINVAL, "bang_build_shard_graph: base or adj is memory of another GPU");
    if (bang::pointer_kind(centres, device) != 0 || (shard_of && bang::pointer_kind(shard_of, device) != 0))
        return sfail(BANG_EINVAL, "bang_build_shard_graph: centres and shard_of must be host memory");
    int prev = -1;
    cudaGetDevice(&prev);
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return sfail(BANG_ECUDA, "bang_build_shard_graph: cannot select the device");
    }
    struct Restore { int d; ~Restore() { if (d >= 0) cudaSetDevice(d); } } restore{prev};
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const uint32_t esz = dtype == BANG_F32 ? 4u : 1u;
    const uint32_t row_bytes = d * esz;
    const uint32_t vbytes = (row_bytes + 15u) & ~15u;
    const uint32_t vwords = vbytes / 4u;
    const uint32_t rec_bytes = (R * 4u + vbytes + 31u) & ~31u;
    const uint32_t rec_words = rec_bytes / 4u;
    const uint64_t nv = n * ell;

    // ---- 1. assignment and shard entries (device)
    DBuf<unsigned char> dX;
    const unsigned char *X = static_cast<const unsigned char *>(base);
    if (bang::pointer_kind(base, device) == 0) {
        SG_TRY(dX.alloc(n * row_bytes));
        SG_TRY(cudaMemcpyAsync(dX.p, base, n * row_bytes, cudaMemcpyHostToDevice, st));
        X = dX.p;
    }
    DBuf<float> dC, dshd;
    DBuf<uint32_t> dsh;
    DBuf<unsigned long long> dekey;
    SG_TRY(dC.alloc(static_cast<uint64_t>(S) * d));
    SG_TRY(cudaMemcpyAsync(dC.p, centres, sizeof(float) * S * d, cudaMemcpyHostToDevice, st));
    SG_TRY(dsh.alloc(nv));
    SG_TRY(dshd.alloc(nv));
    SG_TRY(dekey.alloc(S));
    SG_TRY(cudaMemsetAsync(dekey.p, 0xFF, sizeof(unsigned long long) * S, st));
    if (dtype == BANG_U8) assign_kernel<0><<<blocks(n, 128), 128, 0, st>>>(X, n, d, dC.p, S, ell, dsh.p, dshd.p);
    else if (dtype == BANG_I8) assign_kernel<1><<<blocks(n, 128), 128, 0, st>>>(X, n, d, dC.p, S, ell, dsh.p, dshd.p);
    else assign_kernel<2><<<blocks(n, 128), 128, 0, st>>>(X, n, d, dC.p, S, ell, dsh.p, dshd.p);
    entry_kernel<<<blocks(nv, 256), 256, 0, st>>>(dsh.p, dshd.p, nv, ell, dekey.p);
    SG_TRY(cudaGetLastError());
    std::vector<uint32_t> sh(nv);
    std::vector<unsigned long long> ekey(S);
    SG_TRY(cudaMemcpyAsync(sh.data(), dsh.p, sizeof(uint32_t) * nv, cudaMemcpyDeviceToHost, st));
    SG_TRY(cudaMemcpyAsync(ekey.data(), dekey.p, sizeof(unsigned long long) * S, cudaMemcpyDeviceToHost, st));
    SG_TRY(cudaStreamSynchronize(st));
    dshd.release();
    dC.release();
    dekey.release();

    // ---- 2. members per shard (ascending point id), virtual ids, entries
    std::vector<uint64_t> gstart(S + 1, 0), cur(S);
    for (uint64_t k = 0; k < nv; ++k) gstart[sh[k] + 1]++;
    for (uint32_t g = 0; g < S; ++g) gstart[g + 1] += gstart[g];
    for (uint32_t g = 0; g < S; ++g) cur[g] = gstart[g];
    std::vector<uint32_t> vpt(nv), vid(nv);
    for (uint64_t i = 0; i < n; ++i)
        for (uint32_t t = 0; t < ell; ++t) {
            const uint32_t g = sh[i * ell + t];
            vid[i * ell + t] = static_cast<uint32_t>(cur[g]);
            vpt[cur[g]++] = static_cast<uint32_t>(i);
        }
    std::vector<uint32_t> ventry(S, 0), epos(S, 0), cnt(S), cap(S);
    for (uint32_t g = 0; g < S; ++g) {
        cnt[g] = static_cast<uint32_t>(gstart[g + 1] - gstart[g]);
        cap[g] = std::max<uint32_t>(1u, static_cast<uint32_t>(batch_frac * static_cast<float>(cnt[g])));
        if (cnt[g] == 0) continue;
        const uint64_t pe = ekey[g] & 0xFFFFFFFFull;          // entry point id
        uint32_t v = kNo;
        for (uint32_t t = 0; t < ell; ++t)
            if (sh[pe * ell + t] == g) v = vid[pe * ell + t];
        ventry[g] = v;
        epos[g] = static_cast<uint32_t>(v - gstart[g]);
    }
    if (shard_of) std::memcpy(shard_of, sh.data(), sizeof(uint32_t) * nv);
    std::vector<uint32_t>().swap(sh);

    // ---- records (device): rows empty, vectors copied
    DBuf<uint32_t> rec, dvpt, dvid, dventry;
    DBuf<uint64_t> dgstart;
    SG_TRY(rec.alloc(nv * rec_words));
    SG_TRY(dvpt.alloc(nv));
    SG_TRY(dvid.alloc(nv));
    SG_TRY(dventry.alloc(S));
    SG_TRY(dgstart.alloc(S + 1));
    SG_TRY(cudaMemcpyAsync(dvpt.p, vpt.data(), sizeof(uint32_t) * nv, cudaMemcpyHostToDevice, st));
    SG_TRY(cudaMemcpyAsync(dvid.p, vid.data(), sizeof(uint32_t) * nv, cudaMemcpyHostToDevice, st));
    SG_TRY(cudaMemcpyAsync(dventry.p, ventry.data(), sizeof(uint32_t) * S, cudaMemcpyHostToDevice, st));
    SG_TRY(cudaMemcpyAsync(dgstart.p, gstart.data(), sizeof(uint64_t) * (S + 1), cudaMemcpyHostToDevice, st));
    records_init<<<blocks(nv * rec_words, 256), 256, 0, st>>>(rec.p, nv, rec_words, R, R, X, row_bytes, dvpt.p);
    SG_TRY(cudaGetLastError());
    SG_TRY(cudaStreamSynchronize(st));
    dX.release();

    // ---- 3. two passes of batched insertion
    const uint32_t max_round = [&] {
        uint64_t m = 0;
        for (uint32_t g = 0; g < S; ++g) m += cap[g];
        return static_cast<uint32_t>(std::min<uint64_t>(m, nv));
    }();
    const uint32_t chunk = std::min<uint32_t>(kChunk, std::max<uint32_t>(max_round, 1u));
    DBuf<uint32_t> dseq, qbuf, ebuf, tbuf, ibuf, oid, staging, cntv, tpos, touched, tcnt, fill, in_src;
    DBuf<float> odist;
    DBuf<uint64_t> toff, bsum;
    DBuf<unsigned int> ntouched;
    BigScratch bs;
    SG_TRY(dseq.alloc(nv));
    SG_TRY(qbuf.alloc(static_cast<uint64_t>(chunk) * vwords));   // rows of row_bytes <= vwords * 4
    SG_TRY(ebuf.alloc(chunk));
    SG_TRY(tbuf.alloc(static_cast<uint64_t>(chunk) * iter_cap));
    SG_TRY(ibuf.alloc(chunk));
    SG_TRY(oid.alloc(chunk));
    SG_TRY(odist.alloc(chunk));
    SG_TRY(staging.alloc(static_cast<uint64_t>(max_round) * R));
    SG_TRY(cntv.alloc(nv));
    SG_TRY(tpos.alloc(nv));
    SG_TRY(touched.alloc(std::min<uint64_t>(nv, static_cast<uint64_t>(max_round) * R)));
    SG_TRY(tcnt.alloc(std::min<uint64_t>(nv, static_cast<uint64_t>(max_round) * R)));
    SG_TRY(fill.alloc(std::min<uint64_t>(nv, static_cast<uint64_t>(max_round) * R)));
    SG_TRY(toff.alloc(std::min<uint64_t>(nv, static_cast<uint64_t>(max_round) * R)));
    SG_TRY(in_src.alloc(static_cast<uint64_t>(max_round) * R));
    SG_TRY(ntouched.alloc(1));
    SG_TRY(bs.ndefer.alloc(1));
    SG_TRY(cudaMemsetAsync(cntv.p, 0, sizeof(uint32_t) * nv, st));

    bang::SearchArgs sa;
    std::memset(&sa, 0, sizeof sa);
    sa.adj = rec.p;
    sa.adj_row_words = R;
    sa.adj_stride = rec_words;
    sa.base = rec.p + R;
    sa.vstride = rec_bytes / esz;
    sa.n = static_cast<uint32_t>(nv);
    sa.d = d; sa.M = 1; sa.Mpad = 16; sa.R = R; sa.medoid = 0;
    sa.k = 1; sa.L = Lb; sa.log2z = log2z; sa.iter_cap = iter_cap;
    sa.vec_ok = d % 4 == 0 ? 1u : 0u;              // 4-element loads stay inside aligned rows
    sa.vecb_ok = d % 4 == 0 ? 1u : 0u;
    sa.trace_cap = iter_cap;
    const bang::SmemLayout lay(1, log2z, Lb, 1, d, R, bang::kModeExact);

    LArgs la;
    std::memset(&la, 0, sizeof la);
    la.rec = rec.p; la.recw = rec.p; la.rec_words = rec_words; la.vec_off = R; la.vwords = vwords;
    la.dtype = static_cast<int>(dtype); la.d = d; la.R = R; la.ell = ell;

    std::vector<uint32_t> seq;
    seq.reserve(nv);
    std::vector<uint64_t> roff;
    for (int pass = 0; pass < 2; ++pass) {
        const float a = pass == 0 ? 1.0f : alpha;
        la.a2 = a * a;
        // the pass's insertion sequence, round by round
        seq.clear();
        roff.assign(1, 0);
        std::vector<uint32_t> next(S, 0);
        for (uint32_t r = 0;; ++r) {
            bool any = false;
            for (uint32_t g = 0; g < S; ++g) {
                uint32_t size = pass == 0 ? (r == 0 ? 1u : (r - 1 < 31 ? (1u << (r - 1)) : cap[g])) : cap[g];
                size = std::min(size, cap[g]);
                for (uint32_t e = 0; e < size && next[g] < cnt[g]; ++e, ++next[g]) {
                    const uint32_t pos = next[g];
                    const uint32_t idx = pos == 0 ? epos[g] : (pos - 1 < epos[g] ? pos - 1 : pos);
                    seq.push_back(static_cast<uint32_t>(gstart[g] + idx));
                    any = true;
                }
            }
            if (!any) break;
            roff.push_back(seq.size());
        }
        SG_TRY(cudaMemcpyAsync(dseq.p, seq.data(), sizeof(uint32_t) * seq.size(), cudaMemcpyHostToDevice, st));
        for (size_t r = 0; r + 1 < roff.size(); ++r) {
            const uint32_t *mem = dseq.p + roff[r];
            const uint32_t rn = static_cast<uint32_t>(roff[r + 1] - roff[r]);
            // searches and forward lists, chunk by chunk, into staging
            for (uint32_t c0 = 0; c0 < rn; c0 += chunk) {
                const uint32_t cn = std::min(chunk, rn - c0);
                gather_queries<<<blocks(static_cast<uint64_t>(cn) * row_bytes, 256), 256, 0, st>>>(
                    mem + c0, cn, rec.p, rec_words, R, row_bytes, dgstart.p, S, dventry.p,
                    reinterpret_cast<unsigned char *>(qbuf.p), ebuf.p);
                SG_TRY(cudaGetLastError());
                sa.queries = qbuf.p;
                sa.entry = ebuf.p;
                sa.nq = cn;
                sa.out_ids = oid.p;
                sa.out_dist = odist.p;
                sa.out_iters = ibuf.p;
                sa.trace = tbuf.p;
                SG_TRY(bang::launch_search_exact(sa, static_cast<int>(dtype), lay.total, st));
                la.kind = kJobFwd;
                la.always_prune = 1;
                la.njobs = cn;
                la.members = mem + c0;
                la.trace = tbuf.p;
                la.iters = ibuf.p;
                la.tcap = iter_cap;
                la.staging = staging.p + static_cast<uint64_t>(c0) * R;
                SG_TRY(run_lists(la, bs, st));
            }
            commit_rows<<<blocks(static_cast<uint64_t>(rn) * R, 256), 256, 0, st>>>(mem, rn, staging.p, R, rec.p,
                                                                                 rec_words);
            // reverse edges
            SG_TRY(cudaMemsetAsync(ntouched.p, 0, 4, st));
            rev_count<<<blocks(static_cast<uint64_t>(rn) * R, 256), 256, 0, st>>>(staging.p, rn, R, cntv.p, tpos.p,
                                                                               touched.p, ntouched.p);
            SG_TRY(cudaGetLastError());
            uint32_t nt = 0;
            SG_TRY(cudaMemcpyAsync(&nt, ntouched.p, 4, cudaMemcpyDeviceToHost, st));
            SG_TRY(cudaStreamSynchronize(st));
            if (nt == 0) continue;
            rev_counts_of_touched<<<blocks(nt, 256), 256, 0, st>>>(touched.p, nt, cntv.p, tcnt.p);
            SG_TRY(scan_counts(tcnt.p, nt, toff.p, bsum, st));
            SG_TRY(cudaMemsetAsync(fill.p, 0, sizeof(uint32_t) * nt, st));
            rev_place<<<blocks(static_cast<uint64_t>(rn) * R, 256), 256, 0, st>>>(staging.p, mem, rn, R, tpos.p,
                                                                               toff.p, fill.p, in_src.p);
            SG_TRY(cudaGetLastError());
            la.kind = kJobRev;
            la.always_prune = 0;
            la.njobs = nt;
            la.touched = touched.p;
            la.in_off = toff.p;
            la.in_cnt = tcnt.p;
            la.in_src = in_src.p;
            SG_TRY(run_lists(la, bs, st));
            rev_reset<<<blocks(nt, 256), 256, 0, st>>>(touched.p, nt, cntv.p);
            SG_TRY(cudaGetLastError());
        }
    }
    // free what the merge does not need
    for (auto *b : {&qbuf, &ebuf, &tbuf, &ibuf, &oid, &staging, &cntv, &tpos, &touched, &tcnt, &fill, &in_src, &dseq})
        b->release();
    odist.release();
    toff.release();

    // ---- 4. merge, in chunks of points
    const bool adj_dev = bang::pointer_kind(adj, device) == 1;
    const uint64_t mchunk = std::min<uint64_t>(n, 1ull << 24);
    DBuf<uint32_t> rows;
    if (!adj_dev) SG_TRY(rows.alloc(mchunk * R));
    la.kind = kJobMerge;
    la.always_prune = 0;
    la.a2 = alpha * alpha;
    la.vid = dvid.p;
    la.vpt = dvpt.p;
    for (uint64_t p0 = 0; p0 < n; p0 += mchunk) {
        const uint64_t pn = std::min(mchunk, n - p0);
        la.p0 = p0;
        la.njobs = static_cast<uint32_t>(pn);
        la.out_rows = adj_dev ? adj + p0 * R : rows.p;
        SG_TRY(run_lists(la, bs, st));
        if (!adj_dev)
            SG_TRY(cudaMemcpyAsync(adj + p0 * R, rows.p, sizeof(uint32_t) * pn * R, cudaMemcpyDeviceToHost, st));
    }
    SG_TRY(cudaStreamSynchronize(st));
    return BANG_OK;
}
