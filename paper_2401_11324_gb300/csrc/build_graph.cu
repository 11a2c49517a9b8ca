// GPU build of the clustered graph the large synthetic indexes use (the
// paper searches a graph it takes from DiskANN, §1, and gives no
// construction).  Per cluster (members in ascending id, local position b):
//  1. the K = min(2 Rin, m - 1) members nearest to each member a, by
//     (distance, b), Rin = R - nx;
//  2. RobustPrune (Vamana, §2.2) over them: in (distance, b) order a live
//     candidate is kept (up to Rin) and removes every later candidate j with
//     alpha^2 * d(kept, j) <= d(a, j), alpha^2 and the product in FP32;
//  3. the kept list plus the members that kept a, pruned again;
//  4. repair, members in ascending b: a member nobody links to is appended to
//     the first of its neighbours with room, or replaces that neighbour's
//     last entry if the entry's target keeps another in-link;
//  5. global rows: the list (a cluster medoid keeps at most R - nh), then
//     links to other clusters' medoids, repeats dropped, 0xFFFFFFFF padding.
// Distances are squared L2 rounded to FP32: exact integers for u8/i8
// (converted to FP32), FP32 sums in ascending j for f32 (difference,
// product and sum each rounded).  With that order every step is
// deterministic, so the result does not depend on thread scheduling.
//
// One warp per member for steps 1-3 (a candidate per lane; the nearest K
// kept sorted across the warp's registers, eight per lane); step 4 is
// sequential within a cluster (one thread per cluster); step 5 one warp per
// member.  Vectors are copied to the device with rows padded to 16 bytes
// (int8 stored offset by 128 so that byte differences are unsigned).
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "bang.h"
#include "bang_internal.h"

namespace {

constexpr uint32_t kNo = 0xFFFFFFFFu;
constexpr int kW = 32;
constexpr int kKPL = 8;                 // nearest-candidate keys per lane: K <= 256
constexpr int kWarpsPerBlock = 8;
constexpr uint32_t kMaxRow = 2048;      // padded row bytes (d <= 512 f32, 2048 u8/i8)

struct GArgs {
    const uint4 *X;          // n rows of `stride` 16-byte words
    uint32_t stride;         // 16-byte words per row
    int dtype;               // 0 u8, 1 i8 (stored offset by 128), 2 f32
    uint32_t d;
    const uint32_t *members; // n: ids grouped by cluster
    const uint64_t *gstart;  // ng + 1
    const uint32_t *gof;     // n: cluster of each position
    uint32_t ng, R, Rin, nx, nh;
    float a2;                // alpha^2 in FP32
    const uint32_t *medoids, *xclu, *hclu;
    uint32_t *fwd, *deg;     // n x Rin local positions, n
    uint32_t *fwd2, *deg2;
    uint32_t *rcount, *rfill;
    uint64_t *rstart;        // n + 1
    uint32_t *rsrc;
    uint64_t *scratch;       // per warp slot: union candidate keys
    uint64_t scratch_per_warp;
    uint32_t *indeg;
    uint32_t *adj;           // n x R output (device)
    uint64_t n;
};

// Squared distance between a row held in shared memory (q, `stride` words)
// and a row in global memory, rounded to FP32 as described above.
__device__ __forceinline__ float row_dist(const GArgs &g, const uint4 *q, uint64_t row)
{
    const uint4 *x = g.X + row * g.stride;
    if (g.dtype == 2) {
        float acc = 0.0f;
        uint32_t j = 0;
        for (uint32_t w = 0; w < g.stride && j < g.d; ++w) {
            const uint4 a = q[w], b = __ldg(x + w);
            const float av[4] = {__uint_as_float(a.x), __uint_as_float(a.y), __uint_as_float(a.z),
                                 __uint_as_float(a.w)};
            const float bv[4] = {__uint_as_float(b.x), __uint_as_float(b.y), __uint_as_float(b.z),
                                 __uint_as_float(b.w)};
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                if (j < g.d) {
                    const float t = __fsub_rn(av[i], bv[i]);
                    acc = __fadd_rn(acc, __fmul_rn(t, t));
                }
                ++j;
            }
        }
        return acc;
    }
    uint32_t acc = 0;               // padding bytes are equal on both sides
    for (uint32_t w = 0; w < g.stride; ++w) {
        const uint4 a = q[w], b = __ldg(x + w);
        uint32_t t;
        t = __vabsdiffu4(a.x, b.x); acc = __dp4a(t, t, acc);
        t = __vabsdiffu4(a.y, b.y); acc = __dp4a(t, t, acc);
        t = __vabsdiffu4(a.z, b.z); acc = __dp4a(t, t, acc);
        t = __vabsdiffu4(a.w, b.w); acc = __dp4a(t, t, acc);
    }
    return __uint2float_rn(acc);
}

__device__ __forceinline__ uint64_t mkkey(float dist, uint32_t b)
{
    return (static_cast<uint64_t>(__float_as_uint(dist)) << 32) | b;
}
__device__ __forceinline__ float kdist(uint64_t k) { return __uint_as_float(static_cast<uint32_t>(k >> 32)); }
__device__ __forceinline__ uint32_t kpos(uint64_t k) { return static_cast<uint32_t>(k); }

__device__ __forceinline__ void load_row(const GArgs &g, uint64_t row, uint4 *dst, int lane)
{
    for (uint32_t w = lane; w < g.stride; w += kW) dst[w] = __ldg(g.X + row * g.stride + w);
    __syncwarp();
}

__device__ __forceinline__ uint64_t warp_min64(uint64_t v)
{
    const uint32_t hi = __reduce_min_sync(0xFFFFFFFFu, static_cast<uint32_t>(v >> 32));
    const uint32_t lo = __reduce_min_sync(0xFFFFFFFFu, static_cast<uint32_t>(v >> 32) == hi
                                                           ? static_cast<uint32_t>(v) : 0xFFFFFFFFu);
    return (static_cast<uint64_t>(hi) << 32) | lo;
}

// RobustPrune over the candidate keys keys[0..nc) (any order): repeatedly keep
// the smallest live key and remove the live keys it dominates.  keys live in
// `buf` (nc entries, any memory the warp owns); `qrow` is shared scratch
// for the kept candidate's row.  Writes the kept local positions to out.
__device__ uint32_t prune_keys(const GArgs &g, const uint32_t *P, uint64_t *buf, uint32_t nc,
                               uint32_t Rin, uint32_t *out, uint4 *qrow, int lane)
{
    uint32_t nout = 0;
    const uint64_t kDead = ~0ull;
    while (nout < Rin) {
        uint64_t best = kDead;
        for (uint32_t i = lane; i < nc; i += kW) best = buf[i] < best ? buf[i] : best;
        best = warp_min64(best);
        if (best == kDead) break;
        const uint32_t bk = kpos(best);
        if (lane == 0) out[nout] = bk;
        ++nout;
        load_row(g, P[bk], qrow, lane);
        for (uint32_t i = lane; i < nc; i += kW) {
            const uint64_t k = buf[i];
            if (k == kDead) continue;
            if (k == best) { buf[i] = kDead; continue; }
            const float dij = row_dist(g, qrow, P[kpos(k)]);
            if (__fmul_rn(g.a2, dij) <= kdist(k)) buf[i] = kDead;
        }
        __syncwarp();
    }
    return nout;
}

// Steps 1-2: nearest candidates and the first prune, one warp per member.
__global__ void __launch_bounds__(kW * kWarpsPerBlock) forward_lists(const GArgs g)
{
    __shared__ uint4 rows[kWarpsPerBlock][2][kMaxRow / 16];
    __shared__ uint64_t keys[kWarpsPerBlock][kKPL * kW];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const uint64_t nwarps = static_cast<uint64_t>(gridDim.x) * kWarpsPerBlock;
    for (uint64_t p = static_cast<uint64_t>(blockIdx.x) * kWarpsPerBlock + wib; p < g.n; p += nwarps) {
        const uint32_t c = g.gof[p];
        const uint64_t lo = g.gstart[c];
        const uint32_t m = static_cast<uint32_t>(g.gstart[c + 1] - lo);
        const uint32_t a = static_cast<uint32_t>(p - lo);
        const uint32_t *P = g.members + lo;
        const uint32_t K = 2 * g.Rin < m - 1 ? 2 * g.Rin : m - 1;
        uint4 *qa = rows[wib][0];
        load_row(g, P[a], qa, lane);
        // the nearest K, sorted, entries 8l..8l+7 in lane l
        uint64_t top[kKPL];
#pragma unroll
        for (int i = 0; i < kKPL; ++i) top[i] = ~0ull;
        uint32_t cnt = 0;
        uint64_t thr = ~0ull;            // key of entry K-1 once K are held
        for (uint32_t b0 = 0; b0 < m; b0 += kW) {
            const uint32_t b = b0 + lane;
            uint64_t key = ~0ull;
            if (b < m && b != a) key = mkkey(row_dist(g, qa, P[b]), b);
            uint32_t want = __ballot_sync(0xFFFFFFFFu, key < thr);
            while (want) {
                const int src = __ffs(want) - 1;
                want &= want - 1;
                const uint64_t x = __shfl_sync(0xFFFFFFFFu, key, src);
                if (x >= thr) continue;
                uint32_t below = 0;
#pragma unroll
                for (int i = 0; i < kKPL; ++i) below += top[i] < x ? 1u : 0u;
                const uint32_t pos = __reduce_add_sync(0xFFFFFFFFu, below);
                const uint64_t carry = __shfl_up_sync(0xFFFFFFFFu, top[kKPL - 1], 1);
#pragma unroll
                for (int i = kKPL - 1; i >= 0; --i) {
                    const uint32_t idx = static_cast<uint32_t>(lane) * kKPL + i;
                    const uint64_t prev = i > 0 ? top[i - 1] : (lane > 0 ? carry : ~0ull);
                    if (idx > pos) top[i] = prev;
                    else if (idx == pos) top[i] = x;
                }
                cnt = cnt + 1 < K ? cnt + 1 : K;
                if (cnt == K) {                 // entry K-1: lane (K-1)/8, slot (K-1)%8
                    uint64_t v = 0;
#pragma unroll
                    for (int i = 0; i < kKPL; ++i)
                        if (static_cast<uint32_t>(i) == (K - 1) % kKPL) v = top[i];
                    thr = __shfl_sync(0xFFFFFFFFu, v, (K - 1) / kKPL);
                }
            }
        }
        // entries beyond K are not candidates
        uint64_t *buf = keys[wib];
#pragma unroll
        for (int i = 0; i < kKPL; ++i) {
            const uint32_t idx = static_cast<uint32_t>(lane) * kKPL + i;
            buf[idx] = idx < K ? top[i] : ~0ull;
        }
        __syncwarp();
        uint32_t *out = g.fwd + p * g.Rin;
        const uint32_t nk = prune_keys(g, P, buf, K, g.Rin, out, rows[wib][1], lane);
        if (lane == 0) g.deg[p] = nk;
        __syncwarp();
    }
}

// Reverse edges: counts, then (after the scan) the sources.
__global__ void reverse_count(const GArgs g)
{
    for (uint64_t e = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; e < g.n * g.Rin;
         e += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
        const uint64_t p = e / g.Rin;
        const uint32_t t = static_cast<uint32_t>(e % g.Rin);
        if (t >= g.deg[p]) continue;
        const uint64_t q = g.gstart[g.gof[p]] + g.fwd[e];
        atomicAdd(g.rcount + q, 1u);
    }
}

__global__ void reverse_fill(const GArgs g)
{
    for (uint64_t e = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; e < g.n * g.Rin;
         e += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
        const uint64_t p = e / g.Rin;
        const uint32_t t = static_cast<uint32_t>(e % g.Rin);
        if (t >= g.deg[p]) continue;
        const uint64_t lo = g.gstart[g.gof[p]];
        const uint64_t q = lo + g.fwd[e];
        const uint32_t slot = atomicAdd(g.rfill + q, 1u);
        g.rsrc[g.rstart[q] + slot] = static_cast<uint32_t>(p - lo);
    }
}

// Exclusive scan of n counts into rstart (n + 1): block sums, one block over
// the block sums, then each block's prefix.
constexpr int kScanT = 1024, kScanItems = 4;
__global__ void scan_blocks(const uint32_t *in, uint64_t n, uint64_t *bsum)
{
    __shared__ uint64_t s[kScanT];
    const uint64_t base = static_cast<uint64_t>(blockIdx.x) * kScanT * kScanItems;
    uint64_t v = 0;
    for (int i = 0; i < kScanItems; ++i) {
        const uint64_t k = base + static_cast<uint64_t>(threadIdx.x) * kScanItems + i;
        v += k < n ? in[k] : 0u;
    }
    s[threadIdx.x] = v;
    __syncthreads();
    for (int h = kScanT / 2; h > 0; h >>= 1) {
        if (static_cast<int>(threadIdx.x) < h) s[threadIdx.x] += s[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) bsum[blockIdx.x] = s[0];
}

__global__ void scan_sums(uint64_t *bsum, uint32_t nb)
{
    __shared__ uint64_t s[kScanT];
    uint64_t run = 0;
    for (uint32_t b0 = 0; b0 < nb; b0 += kScanT) {
        const uint32_t i = b0 + threadIdx.x;
        const uint64_t v = i < nb ? bsum[i] : 0;
        s[threadIdx.x] = v;
        __syncthreads();
        for (int h = 1; h < kScanT; h <<= 1) {
            uint64_t add = static_cast<int>(threadIdx.x) >= h ? s[threadIdx.x - h] : 0;
            __syncthreads();
            s[threadIdx.x] += add;
            __syncthreads();
        }
        if (i < nb) bsum[i] = run + s[threadIdx.x] - v;       // exclusive
        run += s[kScanT - 1];
        __syncthreads();
    }
}

__global__ void scan_finish(const uint32_t *in, uint64_t n, const uint64_t *bsum, uint64_t *out)
{
    __shared__ uint64_t s[kScanT];
    const uint64_t base = static_cast<uint64_t>(blockIdx.x) * kScanT * kScanItems;
    uint64_t loc[kScanItems], v = 0;
    for (int i = 0; i < kScanItems; ++i) {
        const uint64_t k = base + static_cast<uint64_t>(threadIdx.x) * kScanItems + i;
        loc[i] = k < n ? in[k] : 0u;
        v += loc[i];
    }
    s[threadIdx.x] = v;
    __syncthreads();
    for (int h = 1; h < kScanT; h <<= 1) {
        uint64_t add = static_cast<int>(threadIdx.x) >= h ? s[threadIdx.x - h] : 0;
        __syncthreads();
        s[threadIdx.x] += add;
        __syncthreads();
    }
    uint64_t run = bsum[blockIdx.x] + s[threadIdx.x] - v;
    for (int i = 0; i < kScanItems; ++i) {
        const uint64_t k = base + static_cast<uint64_t>(threadIdx.x) * kScanItems + i;
        if (k < n) out[k] = run;
        run += loc[i];
        if (k + 1 == n) out[n] = run;
    }
}

// Step 3: the union of the kept list and the reverse sources, pruned again.
__global__ void __launch_bounds__(kW * kWarpsPerBlock) union_lists(const GArgs g)
{
    __shared__ uint4 rows[kWarpsPerBlock][2][kMaxRow / 16];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const uint64_t slot = static_cast<uint64_t>(blockIdx.x) * kWarpsPerBlock + wib;
    const uint64_t nwarps = static_cast<uint64_t>(gridDim.x) * kWarpsPerBlock;
    uint64_t *buf = g.scratch + slot * g.scratch_per_warp;
    for (uint64_t p = slot; p < g.n; p += nwarps) {
        const uint32_t c = g.gof[p];
        const uint64_t lo = g.gstart[c];
        const uint32_t *P = g.members + lo;
        const uint32_t a = static_cast<uint32_t>(p - lo);
        uint4 *qa = rows[wib][0];
        load_row(g, P[a], qa, lane);
        const uint32_t dg = g.deg[p];
        const uint32_t *f = g.fwd + p * g.Rin;
        uint32_t nc = 0;
        for (uint32_t t0 = 0; t0 < dg; t0 += kW) {
            const uint32_t t = t0 + lane;
            if (t < dg) buf[t] = mkkey(row_dist(g, qa, P[f[t]]), f[t]);
        }
        nc = dg;
        const uint64_t r0 = g.rstart[p], r1 = g.rstart[p + 1];
        for (uint64_t r = r0; r < r1; r += kW) {
            const uint64_t ri = r + lane;
            bool add = false;
            uint32_t b = 0;
            if (ri < r1) {
                b = g.rsrc[ri];
                add = true;
                for (uint32_t t = 0; t < dg; ++t) add = add && f[t] != b;
            }
            const uint32_t bal = __ballot_sync(0xFFFFFFFFu, add);
            if (add) buf[nc + __popc(bal & ((1u << lane) - 1u))] = mkkey(row_dist(g, qa, P[b]), b);
            nc += __popc(bal);
        }
        __syncwarp();
        const uint32_t nk = prune_keys(g, P, buf, nc, g.Rin, g.fwd2 + p * g.Rin, rows[wib][1], lane);
        if (lane == 0) g.deg2[p] = nk;
        __syncwarp();
    }
}

__global__ void count_indeg(const GArgs g)
{
    for (uint64_t e = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; e < g.n * g.Rin;
         e += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
        const uint64_t p = e / g.Rin;
        const uint32_t t = static_cast<uint32_t>(e % g.Rin);
        if (t >= g.deg2[p]) continue;
        atomicAdd(g.indeg + g.gstart[g.gof[p]] + g.fwd2[e], 1u);
    }
}

// Step 4: one thread per cluster, members in ascending position.
__global__ void repair(const GArgs g)
{
    const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.ng) return;
    const uint64_t lo = g.gstart[c];
    const uint32_t m = static_cast<uint32_t>(g.gstart[c + 1] - lo);
    for (uint32_t a = 0; a < m; ++a) {
        const uint64_t p = lo + a;
        if (g.indeg[p] != 0 || g.deg2[p] == 0) continue;
        for (uint32_t t = 0; t < g.deg2[p]; ++t) {
            const uint64_t j = lo + g.fwd2[p * g.Rin + t];
            uint32_t *lj = g.fwd2 + j * g.Rin;
            const uint32_t dj = g.deg2[j];
            if (dj < g.Rin) {
                lj[dj] = a;
                g.deg2[j] = dj + 1;
                g.indeg[p] += 1;
                break;
            }
            const uint64_t last = lo + lj[dj - 1];
            if (g.indeg[last] > 1) {
                g.indeg[last] -= 1;
                lj[dj - 1] = a;
                g.indeg[p] += 1;
                break;
            }
        }
    }
}

// Step 5: global rows, one warp per member.
__global__ void __launch_bounds__(kW * kWarpsPerBlock) write_rows(const GArgs g)
{
    __shared__ uint32_t rowbuf[kWarpsPerBlock][256];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const uint64_t nwarps = static_cast<uint64_t>(gridDim.x) * kWarpsPerBlock;
    uint32_t *row = rowbuf[wib];
    for (uint64_t p = static_cast<uint64_t>(blockIdx.x) * kWarpsPerBlock + wib; p < g.n; p += nwarps) {
        const uint32_t c = g.gof[p];
        const uint64_t lo = g.gstart[c];
        const uint32_t *P = g.members + lo;
        const uint32_t a = static_cast<uint32_t>(p - lo);
        const uint32_t pid = P[a];
        const bool is_med = pid == g.medoids[c];
        uint32_t keep = g.deg2[p];
        if (is_med && keep > g.R - g.nh) keep = g.R - g.nh;
        for (uint32_t t = lane; t < keep; t += kW) row[t] = P[g.fwd2[p * g.Rin + t]];
        uint32_t w = keep;
        const uint32_t nl = is_med ? g.nh : g.nx;
        if (lane == 0) {
            for (uint32_t t = 0; t < nl; ++t) {
                const uint32_t c2 = is_med ? g.hclu[static_cast<uint64_t>(c) * g.nh + t]
                                           : g.xclu[static_cast<uint64_t>(pid) * g.nx + t];
                if (c2 >= g.ng || c2 == c || g.medoids[c2] == kNo) continue;
                row[w++] = g.medoids[c2];
            }
        }
        w = __shfl_sync(0xFFFFFFFFu, w, 0);
        __syncwarp();
        // drop repeats (keep the first), then compact
        uint32_t keepmask[8];
#pragma unroll
        for (uint32_t r0 = 0; r0 < 256; r0 += kW) {
            const uint32_t r = r0 + lane;
            bool k = r < w;
            if (k)
                for (uint32_t q = 0; q < r; ++q)
                    if (row[q] == row[r]) { k = false; break; }
            keepmask[r0 / kW] = __ballot_sync(0xFFFFFFFFu, k);
        }
        uint32_t *out = g.adj + static_cast<uint64_t>(pid) * g.R;
        uint32_t before = 0;
#pragma unroll
        for (uint32_t r0 = 0; r0 < 256; r0 += kW) {
            const uint32_t r = r0 + lane, msk = keepmask[r0 / kW];
            if ((msk >> lane) & 1u) out[before + __popc(msk & ((1u << lane) - 1u))] = row[r];
            before += __popc(msk);
        }
        for (uint32_t r = before + lane; r < g.R; r += kW) out[r] = kNo;
        __syncwarp();
    }
}

// Positions -> cluster ids.
__global__ void cluster_of(const uint64_t *gstart, uint32_t ng, uint32_t *gof)
{
    const uint32_t c = blockIdx.x;
    if (c >= ng) return;
    for (uint64_t p = gstart[c] + threadIdx.x; p < gstart[c + 1]; p += blockDim.x) gof[p] = c;
}

// Padded device rows (int8 offset by 128).
__global__ void pad_rows(const uint8_t *src, uint64_t n, uint32_t row_bytes, int dtype,
                         uint32_t stride_bytes, uint8_t *dst)
{
    const uint64_t total = n * stride_bytes;
    for (uint64_t i = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; i < total;
         i += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
        const uint64_t r = i / stride_bytes;
        const uint32_t c = static_cast<uint32_t>(i % stride_bytes);
        uint8_t v = 0;
        if (c < row_bytes) {
            v = src[r * row_bytes + c];
            if (dtype == 1) v ^= 0x80u;
        }
        dst[i] = v;
    }
}

template <typename T> struct DArr {
    T *p = nullptr;
    ~DArr() { if (p) cudaFree(p); }
    cudaError_t alloc(uint64_t count) { return cudaMalloc(&p, sizeof(T) * (count ? count : 1)); }
};

int gfail(int code, const std::string &m)
{
    bang::set_error(m);
    return code;
}

bool is_dev(const void *p)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

template <typename T> cudaError_t to_dev(DArr<T> &d, const T *src, uint64_t count, cudaStream_t st)
{
    cudaError_t e = d.alloc(count);
    if (e != cudaSuccess || count == 0) return e;
    return cudaMemcpyAsync(d.p, src, sizeof(T) * count, cudaMemcpyDefault, st);
}

}  // namespace

#define GB_TRY(x)                                                                           \
    do {                                                                                    \
        cudaError_t e_ = (x);                                                               \
        if (e_ != cudaSuccess) {                                                            \
            cudaGetLastError();                                                             \
            return gfail(e_ == cudaErrorMemoryAllocation ? BANG_ENOMEM : BANG_ECUDA,       \
                         std::string(#x) + ": " + cudaGetErrorString(e_));                  \
        }                                                                                   \
    } while (0)

extern "C" int bang_build_cluster_graph(int device, const void *base, bang_dtype dtype, uint64_t n,
                                        uint32_t d, const uint32_t *members, const uint64_t *gstart,
                                        uint32_t ng, const uint32_t *medoids, uint32_t R, float alpha,
                                        uint32_t nx, const uint32_t *xclu, uint32_t nh,
                                        const uint32_t *hclu, uint32_t *adj, void *stream)
{
    if (!base || !members || !gstart || !medoids || !adj || (nx && !xclu) || (nh && !hclu))
        return gfail(BANG_EINVAL, "bang_build_cluster_graph: NULL argument");
    if (dtype != BANG_U8 && dtype != BANG_I8 && dtype != BANG_F32)
        return gfail(BANG_EINVAL, "bang_build_cluster_graph: unknown dtype");
    if (n == 0 || n >= (1ull << 32) - 1 || d == 0 || ng == 0)
        return gfail(BANG_EINVAL, "bang_build_cluster_graph: need 0 < n < 2^32 - 1, d > 0, ng > 0");
    if (R == 0 || R > 128 || nx >= R || nh >= R || 2 * (R - nx) > kKPL * kW)
        return gfail(BANG_EINVAL, "bang_build_cluster_graph: need R <= 128, nx < R, nh < R");
    const uint32_t esz = dtype == BANG_F32 ? 4u : 1u;
    const uint32_t row_bytes = d * esz, stride_bytes = (row_bytes + 15u) & ~15u;
    if (stride_bytes > kMaxRow) return gfail(BANG_EINVAL, "bang_build_cluster_graph: rows above 2048 bytes");
    if (!(alpha > 0.f)) return gfail(BANG_EINVAL, "bang_build_cluster_graph: alpha must be positive");
    if (bang::pointer_kind(base, device) == 2 || bang::pointer_kind(adj, device) == 2)
        return gfail(BANG_EINVAL, "bang_build_cluster_graph: base or adj is memory of another GPU");
    if (is_dev(members) || is_dev(gstart) || is_dev(medoids) || (nx && is_dev(xclu)) ||
        (nh && is_dev(hclu)))
        return gfail(BANG_EINVAL, "bang_build_cluster_graph: members, gstart, medoids, xclu and hclu "
                     "must be host memory");
    {                   // every id the kernels follow is checked here
        if (gstart[0] != 0 || gstart[ng] != n)
            return gfail(BANG_EINVAL, "bang_build_cluster_graph: gstart must run from 0 to n");
        for (uint32_t c = 0; c < ng; ++c)
            if (gstart[c + 1] < gstart[c])
                return gfail(BANG_EINVAL, "bang_build_cluster_graph: gstart must not decrease");
        std::vector<unsigned char> seen(n, 0);
        for (uint64_t i = 0; i < n; ++i) {
            if (members[i] >= n || seen[members[i]])
                return gfail(BANG_EINVAL, "bang_build_cluster_graph: members must be a permutation of 0..n-1");
            seen[members[i]] = 1;
        }
        for (uint32_t c = 0; c < ng; ++c)
            if (medoids[c] != kNo && medoids[c] >= n)
                return gfail(BANG_EINVAL, "bang_build_cluster_graph: medoid id >= n");
    }
    int prev = -1;
    cudaGetDevice(&prev);
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return gfail(BANG_ECUDA, "bang_build_cluster_graph: cannot select the device");
    }
    struct Restore { int d; ~Restore() { if (d >= 0) cudaSetDevice(d); } } restore{prev};
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    const uint32_t Rin = R - nx;
    DArr<uint8_t> Xraw, Xpad;
    DArr<uint32_t> dmem, dmed, dx, dh, gof, fwd, deg, fwd2, deg2, rcount, rfill, rsrc, indeg, dadj;
    DArr<uint64_t> dgs, rstart, bsum, scratch;
    GB_TRY(Xpad.alloc(n * stride_bytes));
    if (is_dev(base)) {
        pad_rows<<<1024, 256, 0, st>>>(static_cast<const uint8_t *>(base), n, row_bytes, dtype,
                                       stride_bytes, Xpad.p);
    } else {
        GB_TRY(to_dev(Xraw, static_cast<const uint8_t *>(base), n * row_bytes, st));
        pad_rows<<<1024, 256, 0, st>>>(Xraw.p, n, row_bytes, dtype, stride_bytes, Xpad.p);
    }
    GB_TRY(cudaGetLastError());
    GB_TRY(to_dev(dmem, members, n, st));
    GB_TRY(to_dev(dgs, gstart, ng + 1, st));
    GB_TRY(to_dev(dmed, medoids, ng, st));
    GB_TRY(to_dev(dx, xclu, n * nx, st));
    GB_TRY(to_dev(dh, hclu, static_cast<uint64_t>(ng) * nh, st));
    GB_TRY(gof.alloc(n));
    GB_TRY(fwd.alloc(n * Rin));
    GB_TRY(deg.alloc(n));
    GB_TRY(fwd2.alloc(n * Rin));
    GB_TRY(deg2.alloc(n));
    GB_TRY(rcount.alloc(n));
    GB_TRY(rfill.alloc(n));
    GB_TRY(indeg.alloc(n));
    GB_TRY(rstart.alloc(n + 1));
    GB_TRY(rsrc.alloc(n * Rin));
    const bool adj_dev = is_dev(adj);
    if (!adj_dev) GB_TRY(dadj.alloc(n * R));
    GB_TRY(cudaMemsetAsync(rcount.p, 0, n * 4, st));
    GB_TRY(cudaMemsetAsync(rfill.p, 0, n * 4, st));
    GB_TRY(cudaMemsetAsync(indeg.p, 0, n * 4, st));
    cluster_of<<<ng, 256, 0, st>>>(dgs.p, ng, gof.p);

    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    const uint32_t wblocks = static_cast<uint32_t>(sms) * 8u;     // 64 warps per SM
    GArgs g;
    std::memset(&g, 0, sizeof g);
    g.X = reinterpret_cast<const uint4 *>(Xpad.p);
    g.stride = stride_bytes / 16;
    g.dtype = dtype;
    g.d = d;
    g.members = dmem.p;
    g.gstart = dgs.p;
    g.gof = gof.p;
    g.ng = ng;
    g.R = R;
    g.Rin = Rin;
    g.nx = nx;
    g.nh = nh;
    g.a2 = alpha * alpha;
    g.medoids = dmed.p;
    g.xclu = dx.p;
    g.hclu = dh.p;
    g.fwd = fwd.p;
    g.deg = deg.p;
    g.fwd2 = fwd2.p;
    g.deg2 = deg2.p;
    g.rcount = rcount.p;
    g.rfill = rfill.p;
    g.rstart = rstart.p;
    g.rsrc = rsrc.p;
    g.indeg = indeg.p;
    g.adj = adj_dev ? adj : dadj.p;
    g.n = n;

    forward_lists<<<wblocks, kW * kWarpsPerBlock, 0, st>>>(g);
    GB_TRY(cudaGetLastError());
    reverse_count<<<wblocks, 256, 0, st>>>(g);
    const uint32_t nb = static_cast<uint32_t>((n + kScanT * kScanItems - 1) / (kScanT * kScanItems));
    GB_TRY(bsum.alloc(nb));
    scan_blocks<<<nb, kScanT, 0, st>>>(rcount.p, n, bsum.p);
    scan_sums<<<1, kScanT, 0, st>>>(bsum.p, nb);
    scan_finish<<<nb, kScanT, 0, st>>>(rcount.p, n, bsum.p, rstart.p);
    reverse_fill<<<wblocks, 256, 0, st>>>(g);
    GB_TRY(cudaGetLastError());
    // union scratch: the longest candidate list (kept + reverse sources)
    std::vector<uint32_t> cnt(n);
    GB_TRY(cudaMemcpyAsync(cnt.data(), rcount.p, n * 4, cudaMemcpyDeviceToHost, st));
    GB_TRY(cudaStreamSynchronize(st));
    uint64_t maxc = 0;
    for (uint64_t i = 0; i < n; ++i) maxc = cnt[i] > maxc ? cnt[i] : maxc;
    g.scratch_per_warp = maxc + Rin;
    GB_TRY(scratch.alloc(static_cast<uint64_t>(wblocks) * kWarpsPerBlock * g.scratch_per_warp));
    g.scratch = scratch.p;
    union_lists<<<wblocks, kW * kWarpsPerBlock, 0, st>>>(g);
    count_indeg<<<wblocks, 256, 0, st>>>(g);
    repair<<<(ng + 127) / 128, 128, 0, st>>>(g);
    write_rows<<<wblocks, kW * kWarpsPerBlock, 0, st>>>(g);
    GB_TRY(cudaGetLastError());
    if (!adj_dev) GB_TRY(cudaMemcpyAsync(adj, dadj.p, n * R * 4, cudaMemcpyDeviceToHost, st));
    GB_TRY(cudaStreamSynchronize(st));
    return BANG_OK;
}
