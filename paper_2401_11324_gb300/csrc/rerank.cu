// Staged re-rank (§4.8): after the greedy search has converged, the exact
// distances of each query's candidate nodes (the nodes its search expanded,
// recorded by search_kernel when SearchArgs::cand is set) and the k nearest
// of them by (distance, id), as a separate kernel, the way the paper
// structures the step.
//
// One warp per query.  The candidates' vectors are requested U at a time
// (each lane its share of every vector, so U rows are in flight per warp),
// and each distance uses the search kernel's exact-distance arithmetic
// (exact_distance_bits: the same lane shares and the same summation order),
// so the result equals the fused re-rank's bit for bit: both return the k
// smallest (distance, id) keys of the same candidate set.
#include "rerank.h"
#include "search_kernel.cuh"

namespace bang {

namespace {

constexpr int kRerankWarps = 4;      // queries per CTA

template <int DT, int DCH>
__global__ void __launch_bounds__(kRerankWarps * kWarp) rerank_kernel(const RerankArgs a)
{
    using E = typename Elem<DT>::T;
    constexpr int U = DCH == 1 ? 16 : 4;        // candidate vectors requested at once
    __shared__ uint64_t ck_smem[kRerankWarps][kMaxK];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint64_t *Ck = ck_smem[wid];
    const uint32_t kstride = a.k;
    for (uint32_t q = blockIdx.x * kRerankWarps + wid; q < a.nq; q += gridDim.x * kRerankWarps) {
        const uint32_t k = a.k_per_q ? a.k_per_q[q] : a.k;
        const uint32_t L = a.L_per_q ? a.L_per_q[q] : a.L;
        if (k == 0 || k > a.k || L < k || L > a.L) continue;    // padded by the search
        const uint32_t n = a.cand_n[q];
        const uint32_t *cq = a.cand + static_cast<uint64_t>(q) * a.cand_cap;
        VecShare<DT, DCH> qs;
        load_share<DT, DCH>(static_cast<const E *>(a.queries) + static_cast<uint64_t>(q) * a.d, a.d,
                            a.vec_ok != 0, lane, qs);
        const bool regk = k <= static_cast<uint32_t>(kRegK);
        uint64_t ck = ~0ull;             // k <= 32: lane i holds rank i
        uint32_t nc = 0;
        for (uint32_t c0 = 0; c0 < n; c0 += kWarp) {
            const uint32_t mine = c0 + lane < n ? cq[c0 + lane] : kNone;
            const uint32_t cn = n - c0 < static_cast<uint32_t>(kWarp) ? n - c0 : kWarp;
            for (uint32_t j0 = 0; j0 < cn; j0 += U) {
                VecShare<DT, DCH> xs[U];
                uint32_t id[U];
#pragma unroll
                for (int j = 0; j < U; ++j) {
                    id[j] = __shfl_sync(0xFFFFFFFFu, mine, static_cast<int>((j0 + j) & 31u));
                    if (j0 + j < cn)
                        load_share<DT, DCH>(static_cast<const E *>(a.base) + static_cast<uint64_t>(id[j]) * a.vstride,
                                            a.d, a.vecb_ok != 0, lane, xs[j]);
                }
#pragma unroll
                for (int j = 0; j < U; ++j) {
                    if (j0 + j >= cn) break;
                    const uint64_t e = make_key(exact_distance_bits<DT, DCH>(qs, xs[j]), id[j]);
                    if (regk) {
                        const uint32_t pos = __popc(__ballot_sync(0xFFFFFFFFu, ck < e));
                        if (pos < k) {
                            const uint64_t up = shfl_up_u64(ck, 1);
                            if (static_cast<uint32_t>(lane) == pos) ck = e;
                            else if (static_cast<uint32_t>(lane) > pos) ck = up;
                        }
                        nc = nc + 1 < k ? nc + 1 : k;
                    } else if (!(nc == k && e >= Ck[k - 1])) {
                        // rank of e among the kept keys, then shift the larger ones up
                        uint32_t less = 0;
                        uint64_t keep[kMaxK / kWarp];
#pragma unroll
                        for (int t = 0; t < kMaxK / kWarp; ++t) {
                            const uint32_t i = lane + kWarp * t;
                            keep[t] = i < nc ? Ck[i] : 0ull;
                            less += (i < nc && keep[t] < e) ? 1u : 0u;
                        }
                        const uint32_t pos = __reduce_add_sync(0xFFFFFFFFu, less);
                        __syncwarp();
#pragma unroll
                        for (int t = 0; t < kMaxK / kWarp; ++t) {
                            const uint32_t i = lane + kWarp * t;
                            if (i < nc && i >= pos && i + 1 < k) Ck[i + 1] = keep[t];
                        }
                        if (lane == 0) Ck[pos] = e;
                        nc = nc + 1 < k ? nc + 1 : k;
                        __syncwarp();
                    }
                }
            }
        }
        __syncwarp();
        for (uint32_t i = lane; i < kstride; i += kWarp) {
            const uint64_t o = static_cast<uint64_t>(q) * kstride + i;
            uint64_t key = ~0ull;
            if (i < nc) key = regk ? ck : Ck[i];     // regk: nc <= k <= 32, rank i is lane i's
            if (i < nc) {
                const uint32_t bits = static_cast<uint32_t>(key >> 32);
                a.out_ids[o] = key_id(key);
                a.out_dist[o] = DT == 2 ? __uint_as_float(bits) : static_cast<float>(bits);
            } else {
                a.out_ids[o] = kNone;
                a.out_dist[o] = __uint_as_float(0x7F800000u);
            }
        }
        __syncwarp();
    }
}

// 64-bit key exchange across lanes at xor distance j.
__device__ __forceinline__ uint64_t shfl_xor_u64(uint64_t v, int j)
{
    const uint32_t lo = __shfl_xor_sync(0xFFFFFFFFu, static_cast<uint32_t>(v), j);
    const uint32_t hi = __shfl_xor_sync(0xFFFFFFFFu, static_cast<uint32_t>(v >> 32), j);
    return (static_cast<uint64_t>(hi) << 32) | lo;
}

// Ascending bitonic sort of one key per lane (lane i ends with rank i).
__device__ __forceinline__ uint64_t warp_sort_keys(uint64_t v, int lane)
{
#pragma unroll
    for (int size = 2; size <= kWarp; size <<= 1) {
        const bool up = (lane & size) == 0;          // segment sorted ascending
#pragma unroll
        for (int j = size >> 1; j > 0; j >>= 1) {
            const uint64_t o = shfl_xor_u64(v, j);
            const bool keep_min = ((lane & j) == 0) == up;
            v = keep_min ? (o < v ? o : v) : (o > v ? o : v);
        }
    }
    return v;
}

// Integer vectors (u8, int8) with d a multiple of 16 up to 128 and k <= 32:
// exact distances are integer sums, equal in any order, so one lane takes one
// candidate's whole row (up to eight 16-byte loads, 32 rows in flight per
// warp and two batches requested at once); a batch's 32 keys are sorted and
// merged into the running top 32 (lane i holds rank i): the element-wise
// minimum of the top list and the reversed batch holds the 32 smallest keys of
// both as a bitonic sequence, which five exchange steps sort.  The k smallest
// keys of the candidate set come out, as in the warp-per-candidate kernel.
template <int DT>
__global__ void __launch_bounds__(kRerankWarps * kWarp) rerank_lanes_kernel(const RerankArgs a)
{
    __shared__ uint4 qsm[kRerankWarps][8];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const uint32_t kstride = a.k, nw16 = a.d / 16u;
    const uint32_t bias = DT == 1 ? 0x80808080u : 0u;    // int8: bytes biased, differences unsigned
    for (uint32_t q = blockIdx.x * kRerankWarps + wid; q < a.nq; q += gridDim.x * kRerankWarps) {
        const uint32_t k = a.k_per_q ? a.k_per_q[q] : a.k;
        const uint32_t L = a.L_per_q ? a.L_per_q[q] : a.L;
        if (k == 0 || k > a.k || L < k || L > a.L) continue;    // padded by the search
        const uint32_t n = a.cand_n[q];
        const uint32_t *cq = a.cand + static_cast<uint64_t>(q) * a.cand_cap;
        {   // the query's words, biased like the rows (byte loads: any alignment)
            const uint8_t *qb = static_cast<const uint8_t *>(a.queries) + static_cast<uint64_t>(q) * a.d;
            uint32_t w = 0;
            if (static_cast<uint32_t>(lane) * 4u < a.d)
                w = (static_cast<uint32_t>(qb[4 * lane]) | static_cast<uint32_t>(qb[4 * lane + 1]) << 8 |
                     static_cast<uint32_t>(qb[4 * lane + 2]) << 16 | static_cast<uint32_t>(qb[4 * lane + 3]) << 24) ^ bias;
            reinterpret_cast<uint32_t *>(qsm[wid])[lane] = w;
        }
        __syncwarp();
        uint64_t top = ~0ull;
        for (uint32_t c0 = 0; c0 < n; c0 += 2 * kWarp) {
            uint4 row[2][8];
            uint32_t id[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const uint32_t i = c0 + h * kWarp + lane;
                id[h] = i < n ? cq[i] : kNone;
                const uint4 *rp = reinterpret_cast<const uint4 *>(static_cast<const uint8_t *>(a.base) +
                                                                  static_cast<uint64_t>(id[h] == kNone ? 0u : id[h]) * a.vstride);
#pragma unroll
                for (int c = 0; c < 8; ++c)
                    row[h][c] = (id[h] != kNone && static_cast<uint32_t>(c) < nw16) ? __ldg(rp + c)
                                                                                  : make_uint4(0u, 0u, 0u, 0u);
            }
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                if (c0 + h * kWarp >= n) break;                       // warp-uniform
                uint32_t acc = 0;
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    if (static_cast<uint32_t>(c) >= nw16) break;
                    const uint4 qv = qsm[wid][c];
                    const uint32_t xw[4] = {row[h][c].x ^ bias, row[h][c].y ^ bias, row[h][c].z ^ bias,
                                            row[h][c].w ^ bias};
                    const uint32_t qw[4] = {qv.x, qv.y, qv.z, qv.w};
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const uint32_t df = __vabsdiffu4(qw[i], xw[i]);
                        acc = __dp4a(df, df, acc);
                    }
                }
                uint64_t key = id[h] != kNone ? make_key(acc, id[h]) : ~0ull;
                key = warp_sort_keys(key, lane);
                const uint64_t rev = shfl_u64(key, kWarp - 1 - lane);
                uint64_t m = rev < top ? rev : top;
#pragma unroll
                for (int j = kWarp / 2; j > 0; j >>= 1) {
                    const uint64_t o = shfl_xor_u64(m, j);
                    m = (lane & j) == 0 ? (o < m ? o : m) : (o > m ? o : m);
                }
                top = m;
            }
        }
        const uint32_t nc = n < k ? n : k;
        for (uint32_t i = lane; i < kstride; i += kWarp) {
            const uint64_t o = static_cast<uint64_t>(q) * kstride + i;
            if (i < nc) {                   // nc <= k <= 32: rank i is lane i's key
                a.out_ids[o] = key_id(top);
                a.out_dist[o] = static_cast<float>(static_cast<uint32_t>(top >> 32));
            } else {
                a.out_ids[o] = kNone;
                a.out_dist[o] = __uint_as_float(0x7F800000u);
            }
        }
        __syncwarp();
    }
}

template <int DT, int DCH>
cudaError_t launch_dt(const RerankArgs &a, cudaStream_t st)
{
    if constexpr (DT != 2 && DCH == 1) {
        // rows reachable with 16-byte loads; k within one lane per rank
        if (a.d % 16u == 0 && a.k <= static_cast<uint32_t>(kRegK) && a.vecb_ok && a.vstride % 16u == 0) {
            const uint32_t blocks = (a.nq + kRerankWarps - 1) / kRerankWarps;
            rerank_lanes_kernel<DT><<<blocks, kRerankWarps * kWarp, 0, st>>>(a);
            return cudaGetLastError();
        }
    }
    const uint32_t blocks = (a.nq + kRerankWarps - 1) / kRerankWarps;
    rerank_kernel<DT, DCH><<<blocks, kRerankWarps * kWarp, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_rerank(const RerankArgs &a, int dtype, cudaStream_t st)
{
    if (a.nq == 0) return cudaSuccess;
    const bool narrow = a.d <= 128;
    if (dtype == 0) return narrow ? launch_dt<0, 1>(a, st) : launch_dt<0, 4>(a, st);
    if (dtype == 1) return narrow ? launch_dt<1, 1>(a, st) : launch_dt<1, 4>(a, st);
    return narrow ? launch_dt<2, 1>(a, st) : launch_dt<2, 4>(a, st);
}

}  // namespace bang
