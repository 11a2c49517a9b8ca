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

template <int DT, int DCH>
cudaError_t launch_dt(const RerankArgs &a, cudaStream_t st)
{
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
