// Exact k nearest neighbours on the GPU: the ground truth that recall@k
// (§6.3, k-recall@k) is measured against.  Distances are squared L2, exact
// integers for u8/i8 data and FP64 for f32 data, the latter summed in
// ascending dimension order with each difference, product and sum rounded
// (no fused multiply-add); ties go to the smaller id.  The only FP64 on the
// GPU in this library besides the offline k-means.
//
// Three passes.  (1) Each query's exact k nearest among the first S points
// (S = min(n, 262144)) give a threshold: the k-th of them is at least the
// k-th over all n points, so every true neighbour is within it.  (2) A tile
// of queries held in shared memory streams over all points, one point per
// thread, and appends every point within a query's threshold to that query's
// candidate list.  (3) One warp per query picks the k smallest candidates by
// (distance, id).  A list that overflows its capacity is detected and pass 2
// rerun with room for the longest list.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "bang.h"
#include "bang_internal.h"

namespace {

constexpr uint32_t kNo = 0xFFFFFFFFu;
constexpr int kW = 32;
constexpr int kKPL = 8;                  // top-k entries per lane in pass 1: k <= 256
constexpr uint32_t kTileQ = 128;         // at most this many queries per CTA in pass 2
constexpr uint32_t kSample = 262144;

struct GtArgs {
    const void *base, *queries;
    int dtype;
    uint64_t n;
    uint32_t nq, d, k;
    const double *thr;           // nq thresholds (pass 2)
    double *thr_out;             // pass 1
    uint32_t *cnt;               // nq candidate counts
    double *cd;                  // nq x cap candidate distances
    uint32_t *ci;                // nq x cap candidate ids
    uint64_t cap;
    uint32_t *out_ids;
    double *out_dist;
    uint32_t tileq;              // queries per CTA in pass 2 (46 KB of rows at most)
    uint32_t words;              // integer rows readable as 32-bit words (d % 4 == 0, aligned)
    uint32_t regrow;             // integer rows of 16..128 bytes in 16-byte steps, 16-byte aligned
};

// Squared distance of two rows of 32-bit words of packed bytes (int8 offset
// by 128 on both sides, so byte differences are unsigned).
__device__ __forceinline__ uint32_t word_dist(uint32_t a, uint32_t b, uint32_t acc, bool i8)
{
    if (i8) { a ^= 0x80808080u; b ^= 0x80808080u; }
    const uint32_t t = __vabsdiffu4(a, b);
    return __dp4a(t, t, acc);
}

__device__ __forceinline__ double dist_rows(const GtArgs &g, const void *qrow, uint64_t i)
{
    if (g.dtype == 2) {
        const float *q = static_cast<const float *>(qrow);
        const float *x = static_cast<const float *>(g.base) + i * g.d;
        double acc = 0.0;
        for (uint32_t j = 0; j < g.d; ++j) {
            const double t = __dsub_rn(static_cast<double>(q[j]), static_cast<double>(__ldg(x + j)));
            acc = __dadd_rn(acc, __dmul_rn(t, t));
        }
        return acc;
    }
    if (g.words) {
        const uint32_t *q = static_cast<const uint32_t *>(qrow);
        const uint32_t *x = reinterpret_cast<const uint32_t *>(static_cast<const unsigned char *>(g.base) + i * g.d);
        uint32_t acc = 0;       // at most d * 255^2 < 2^32 (d <= 4096)
        for (uint32_t w = 0; w < g.d / 4u; ++w) acc = word_dist(q[w], __ldg(x + w), acc, g.dtype == 1);
        return static_cast<double>(acc);
    }
    int64_t acc = 0;
    if (g.dtype == 0) {
        const uint8_t *q = static_cast<const uint8_t *>(qrow);
        const uint8_t *x = static_cast<const uint8_t *>(g.base) + i * g.d;
        for (uint32_t j = 0; j < g.d; ++j) {
            const int32_t t = static_cast<int32_t>(q[j]) - static_cast<int32_t>(__ldg(x + j));
            acc += t * t;
        }
    } else {
        const int8_t *q = static_cast<const int8_t *>(qrow);
        const int8_t *x = static_cast<const int8_t *>(g.base) + i * g.d;
        for (uint32_t j = 0; j < g.d; ++j) {
            const int32_t t = static_cast<int32_t>(q[j]) - static_cast<int32_t>(__ldg(x + j));
            acc += t * t;
        }
    }
    return static_cast<double>(acc);
}

__device__ __forceinline__ const void *query_row(const GtArgs &g, uint32_t q)
{
    const size_t esz = g.dtype == 2 ? 4 : 1;
    return static_cast<const unsigned char *>(g.queries) + static_cast<uint64_t>(q) * g.d * esz;
}

// (distance, id) order; distances are >= +0, so their bit patterns order like
// their values.
__device__ __forceinline__ bool less_pair(uint64_t da, uint32_t ia, uint64_t db, uint32_t ib)
{
    return da < db || (da == db && ia < ib);
}

// Pass 1: one warp per query, the exact k nearest of the first S points kept
// sorted across the warp (8 per lane); the threshold is the k-th distance.
__global__ void sample_threshold(const GtArgs g, uint64_t S)
{
    const int lane = threadIdx.x & 31;
    const uint32_t q = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (q >= g.nq) return;
    const void *qr = query_row(g, q);
    uint64_t td[kKPL];
    uint32_t ti[kKPL];
#pragma unroll
    for (int t = 0; t < kKPL; ++t) { td[t] = ~0ull; ti[t] = kNo; }
    uint32_t cnt = 0;
    uint64_t thd = ~0ull;
    uint32_t thi = kNo;
    for (uint64_t b0 = 0; b0 < S; b0 += kW) {
        const uint64_t i = b0 + lane;
        uint64_t dk = ~0ull;
        uint32_t ik = kNo;
        if (i < S) {
            dk = static_cast<uint64_t>(__double_as_longlong(dist_rows(g, qr, i)));
            ik = static_cast<uint32_t>(i);
        }
        uint32_t want = __ballot_sync(0xFFFFFFFFu, ik != kNo && less_pair(dk, ik, thd, thi));
        while (want) {
            const int src = __ffs(want) - 1;
            want &= want - 1;
            const uint64_t xd = __shfl_sync(0xFFFFFFFFu, dk, src);
            const uint32_t xi = __shfl_sync(0xFFFFFFFFu, ik, src);
            if (!less_pair(xd, xi, thd, thi)) continue;
            uint32_t below = 0;
#pragma unroll
            for (int t = 0; t < kKPL; ++t) below += less_pair(td[t], ti[t], xd, xi) ? 1u : 0u;
            const uint32_t pos = __reduce_add_sync(0xFFFFFFFFu, below);
            const uint64_t cd = __shfl_up_sync(0xFFFFFFFFu, td[kKPL - 1], 1);
            const uint32_t ci = __shfl_up_sync(0xFFFFFFFFu, ti[kKPL - 1], 1);
#pragma unroll
            for (int t = kKPL - 1; t >= 0; --t) {
                const uint32_t idx = static_cast<uint32_t>(lane) * kKPL + t;
                const uint64_t pd = t > 0 ? td[t - 1] : (lane > 0 ? cd : ~0ull);
                const uint32_t pi = t > 0 ? ti[t - 1] : (lane > 0 ? ci : kNo);
                if (idx > pos) { td[t] = pd; ti[t] = pi; }
                else if (idx == pos) { td[t] = xd; ti[t] = xi; }
            }
            cnt = cnt + 1 < g.k ? cnt + 1 : g.k;
            if (cnt == g.k) {
                uint64_t vd = 0;
                uint32_t vi = 0;
#pragma unroll
                for (int t = 0; t < kKPL; ++t)
                    if (static_cast<uint32_t>(t) == (g.k - 1) % kKPL) { vd = td[t]; vi = ti[t]; }
                thd = __shfl_sync(0xFFFFFFFFu, vd, (g.k - 1) / kKPL);
                thi = __shfl_sync(0xFFFFFFFFu, vi, (g.k - 1) / kKPL);
            }
        }
    }
    if (lane == 0)       // fewer than k sampled points: every point is a candidate
        g.thr_out[q] = cnt == g.k ? __longlong_as_double(static_cast<long long>(thd))
                                  : __longlong_as_double(0x7FF0000000000000ll);
}

// Pass 2: blockIdx.y = tile of kTileQ queries (rows in shared memory);
// threads stride over the points.
__global__ void collect(const GtArgs g)
{
    extern __shared__ __align__(16) unsigned char qs[];
    const uint32_t q0 = blockIdx.y * g.tileq;
    const uint32_t nt = g.nq - q0 < g.tileq ? g.nq - q0 : g.tileq;
    const size_t rowb = static_cast<size_t>(g.d) * (g.dtype == 2 ? 4 : 1);
    for (size_t i = threadIdx.x; i < nt * rowb; i += blockDim.x)
        qs[i] = static_cast<const unsigned char *>(query_row(g, q0))[i];
    __shared__ double th[kTileQ];
    if (threadIdx.x < nt) th[threadIdx.x] = g.thr[q0 + threadIdx.x];
    __syncthreads();
    for (uint64_t i = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; i < g.n;
         i += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
        uint4 xr[8];                     // the point's row, for the register path
        const uint32_t nv = g.d / 16u;
        if (g.regrow) {
            const uint4 *x = reinterpret_cast<const uint4 *>(static_cast<const unsigned char *>(g.base) + i * g.d);
#pragma unroll
            for (int c = 0; c < 8; ++c) xr[c] = static_cast<uint32_t>(c) < nv ? __ldg(x + c) : make_uint4(0u, 0u, 0u, 0u);
        }
        for (uint32_t t = 0; t < nt; ++t) {
            double dv;
            if (g.regrow) {
                const uint4 *qv = reinterpret_cast<const uint4 *>(qs + t * rowb);
                uint32_t acc = 0;
                const bool i8 = g.dtype == 1;
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    if (static_cast<uint32_t>(c) < nv) {
                        const uint4 a = qv[c], b = xr[c];
                        acc = word_dist(a.x, b.x, acc, i8);
                        acc = word_dist(a.y, b.y, acc, i8);
                        acc = word_dist(a.z, b.z, acc, i8);
                        acc = word_dist(a.w, b.w, acc, i8);
                    }
                }
                dv = static_cast<double>(acc);
            } else {
                dv = dist_rows(g, qs + t * rowb, i);
            }
            if (dv <= th[t]) {
                const uint32_t q = q0 + t;
                const uint32_t slot = atomicAdd(g.cnt + q, 1u);
                if (slot < g.cap) {
                    g.cd[static_cast<uint64_t>(q) * g.cap + slot] = dv;
                    g.ci[static_cast<uint64_t>(q) * g.cap + slot] = static_cast<uint32_t>(i);
                }
            }
        }
    }
}

// Pass 3: one warp per query, the k smallest candidates in (distance, id) order.
__global__ void select_k(const GtArgs g)
{
    const int lane = threadIdx.x & 31;
    const uint32_t q = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (q >= g.nq) return;
    const uint64_t m = g.cnt[q] < g.cap ? g.cnt[q] : g.cap;
    const double *cd = g.cd + static_cast<uint64_t>(q) * g.cap;
    const uint32_t *ci = g.ci + static_cast<uint64_t>(q) * g.cap;
    uint64_t pd = 0;             // the last pair taken (exclusive lower bound)
    uint32_t pi = 0;
    bool first = true;
    for (uint32_t r = 0; r < g.k; ++r) {
        uint64_t bd = ~0ull;
        uint32_t bi = kNo;
        for (uint64_t j = lane; j < m; j += kW) {
            const uint64_t dj = static_cast<uint64_t>(__double_as_longlong(cd[j]));
            const uint32_t ij = ci[j];
            if (!first && !less_pair(pd, pi, dj, ij)) continue;          // already taken
            if (less_pair(dj, ij, bd, bi)) { bd = dj; bi = ij; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const uint64_t od = __shfl_xor_sync(0xFFFFFFFFu, bd, o);
            const uint32_t oi = __shfl_xor_sync(0xFFFFFFFFu, bi, o);
            if (less_pair(od, oi, bd, bi)) { bd = od; bi = oi; }
        }
        const uint64_t o = static_cast<uint64_t>(q) * g.k + r;
        if (lane == 0) {
            g.out_ids[o] = bi;
            g.out_dist[o] = bi == kNo ? __longlong_as_double(0x7FF0000000000000ll)
                                      : __longlong_as_double(static_cast<long long>(bd));
        }
        pd = bd;
        pi = bi;
        first = false;
    }
}

template <typename T> struct DArr {
    T *p = nullptr;
    ~DArr() { if (p) cudaFree(p); }
    cudaError_t alloc(uint64_t count)
    {
        if (p) cudaFree(p);
        p = nullptr;
        return cudaMalloc(&p, sizeof(T) * (count ? count : 1));
    }
};

bool is_dev(const void *p)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

int gtfail(int code, const std::string &m)
{
    bang::set_error(m);
    return code;
}

}  // namespace

#define GT_TRY(x)                                                                           \
    do {                                                                                    \
        cudaError_t e_ = (x);                                                               \
        if (e_ != cudaSuccess) {                                                            \
            cudaGetLastError();                                                             \
            return gtfail(e_ == cudaErrorMemoryAllocation ? BANG_ENOMEM : BANG_ECUDA,      \
                          std::string(#x) + ": " + cudaGetErrorString(e_));                 \
        }                                                                                   \
    } while (0)

extern "C" int bang_ground_truth(int device, const void *base, const void *queries, bang_dtype dtype,
                                 uint64_t n, uint32_t nq, uint32_t d, uint32_t k, uint32_t *out_ids,
                                 double *out_dist, void *stream)
{
    if (!base || !queries || !out_ids || !out_dist) return gtfail(BANG_EINVAL, "bang_ground_truth: NULL argument");
    if (dtype != BANG_U8 && dtype != BANG_I8 && dtype != BANG_F32)
        return gtfail(BANG_EINVAL, "bang_ground_truth: unknown dtype");
    if (n == 0 || n >= (1ull << 32) - 1 || d == 0 || d > 4096 || k == 0 || k > kKPL * kW)
        return gtfail(BANG_EINVAL, "bang_ground_truth: need 0 < n < 2^32 - 1, 0 < d <= 4096, 1 <= k <= 256");
    if (bang::pointer_kind(base, device) == 2 || bang::pointer_kind(queries, device) == 2 ||
        bang::pointer_kind(out_ids, device) == 2 || bang::pointer_kind(out_dist, device) == 2)
        return gtfail(BANG_EINVAL, "bang_ground_truth: a buffer is memory of another GPU");
    if (nq == 0) return BANG_OK;
    const size_t esz = dtype == BANG_F32 ? 4 : 1;
    // query rows in dynamic shared memory; with the thresholds (static) under 48 KB
    const uint32_t tileq = static_cast<uint32_t>(std::min<size_t>(kTileQ, (46u * 1024u) / (d * esz)));
    if (tileq == 0) return gtfail(BANG_EINVAL, "bang_ground_truth: rows too long");
    int prev = -1;
    cudaGetDevice(&prev);
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return gtfail(BANG_ECUDA, "bang_ground_truth: cannot select the device");
    }
    struct Restore { int d; ~Restore() { if (d >= 0) cudaSetDevice(d); } } restore{prev};
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    DArr<unsigned char> dbase, dq;
    const void *B = base, *Q = queries;
    if (!is_dev(base)) {
        GT_TRY(dbase.alloc(n * d * esz));
        GT_TRY(cudaMemcpyAsync(dbase.p, base, n * d * esz, cudaMemcpyHostToDevice, st));
        B = dbase.p;
    }
    if (!is_dev(queries)) {
        GT_TRY(dq.alloc(static_cast<uint64_t>(nq) * d * esz));
        GT_TRY(cudaMemcpyAsync(dq.p, queries, static_cast<uint64_t>(nq) * d * esz, cudaMemcpyHostToDevice, st));
        Q = dq.p;
    }
    const uint64_t S = n < kSample ? n : kSample;
    DArr<double> thr, cd, odist;
    DArr<uint32_t> cnt, ci, oids;
    GT_TRY(thr.alloc(nq));
    GT_TRY(cnt.alloc(nq));
    GtArgs g;
    std::memset(&g, 0, sizeof g);
    g.base = B;
    g.queries = Q;
    g.dtype = dtype;
    g.n = n;
    g.nq = nq;
    g.d = d;
    g.k = k;
    g.thr_out = thr.p;
    g.thr = thr.p;
    g.cnt = cnt.p;
    g.tileq = tileq;
    {
        const uintptr_t ab = reinterpret_cast<uintptr_t>(B), aq = reinterpret_cast<uintptr_t>(Q);
        g.words = dtype != BANG_F32 && d % 4 == 0 && ab % 4 == 0 && aq % 4 == 0;
        g.regrow = dtype != BANG_F32 && d % 16 == 0 && d <= 128 && ab % 16 == 0;
    }
    sample_threshold<<<(nq + 3) / 4, 128, 0, st>>>(g, S);
    GT_TRY(cudaGetLastError());
    // expected list length about k * n / S; room for twice that, then the longest
    uint64_t cap = 2ull * k * ((n + S - 1) / S) + 256;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    const uint32_t tiles = (nq + tileq - 1) / tileq;
    const uint32_t gx = static_cast<uint32_t>((static_cast<uint64_t>(sms) * 8 + tiles - 1) / tiles) + 1;
    for (int attempt = 0; attempt < 2; ++attempt) {
        GT_TRY(cd.alloc(cap * nq));
        GT_TRY(ci.alloc(cap * nq));
        GT_TRY(cudaMemsetAsync(cnt.p, 0, nq * 4, st));
        g.cd = cd.p;
        g.ci = ci.p;
        g.cap = cap;
        collect<<<dim3(gx, tiles), 256, tileq * d * esz, st>>>(g);
        GT_TRY(cudaGetLastError());
        std::vector<uint32_t> c(nq);
        GT_TRY(cudaMemcpyAsync(c.data(), cnt.p, nq * 4, cudaMemcpyDeviceToHost, st));
        GT_TRY(cudaStreamSynchronize(st));
        uint64_t mx = 0;
        for (uint32_t i = 0; i < nq; ++i) mx = c[i] > mx ? c[i] : mx;
        if (mx <= cap) break;
        if (attempt == 1) return gtfail(BANG_ECUDA, "bang_ground_truth: candidate lists kept growing");
        cap = mx;
    }
    const bool dev_out = is_dev(out_ids);
    if (!dev_out) {
        GT_TRY(oids.alloc(static_cast<uint64_t>(nq) * k));
        GT_TRY(odist.alloc(static_cast<uint64_t>(nq) * k));
    }
    g.out_ids = dev_out ? out_ids : oids.p;
    g.out_dist = dev_out ? out_dist : odist.p;
    select_k<<<(nq + 3) / 4, 128, 0, st>>>(g);
    GT_TRY(cudaGetLastError());
    if (!dev_out) {
        GT_TRY(cudaMemcpyAsync(out_ids, oids.p, static_cast<uint64_t>(nq) * k * 4, cudaMemcpyDeviceToHost, st));
        GT_TRY(cudaMemcpyAsync(out_dist, odist.p, static_cast<uint64_t>(nq) * k * 8, cudaMemcpyDeviceToHost, st));
    }
    GT_TRY(cudaStreamSynchronize(st));
    return BANG_OK;
}
