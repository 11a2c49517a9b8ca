// Greedy-search kernel of BANG (arXiv 2401.11324), FP32 form, for sm_103a.
//
// One warp (a 32-thread CTA) runs the whole search of one query: the PQ
// distance table (§4.1), the Bloom-filter seen set (§4.3), the worklist and
// the re-rank candidates all live in shared memory, so the only global
// traffic per iteration is the neighbour list and full vector of the expanded
// node (read in place from page-locked host memory, Alg. 2 "FetchNeighbors")
// and one PQ code row per new neighbour (HBM, §4.4).
//
// The paper splits every iteration into separate kernels with one CTA per
// query and keeps the table and filter in global memory; here the iteration
// loop stays inside one CTA, and the eager next-node choice of §4.5 becomes
// a software prefetch: the next node's lists are requested right after the
// distances are known, and arrive while the warp merges the worklist.
//
// Arithmetic order (fixed so that results are reproducible bit for bit):
//  - table entry T[s][c]: fmaf(q_j - C_j, q_j - C_j, acc) over the subspace's
//    dimensions in ascending j, from 0;
//  - PQ distance: eight partial sums over subspaces s = r (mod 8), in
//    ascending s, then p_r += p_(r^4), p_r += p_(r^2), p_r += p_(r^1);
//  - exact distance: 32 partial sums, one per lane, lane r owning the
//    dimensions j with (j/4) mod 32 = r in ascending j (fmaf), then a
//    butterfly over xor distances 16, 8, 4, 2, 1; integer data sums exactly;
//  - ordering keys are (distance, id), distance compared as FP32 (integer
//    exact distances as unsigned integers).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace bang {

constexpr uint32_t kNone = 0xFFFFFFFFu;
constexpr int kWarp = 32;
constexpr int kMaxR = 128;        // neighbours per row: 4 per lane
constexpr int kMaxRPL = kMaxR / kWarp;
constexpr int kMaxD = 512;        // dimensions: 16 per lane for the exact distance
constexpr int kMaxDPL = kMaxD / kWarp;
constexpr int kMaxM = 128;
constexpr int kMaxK = 256;
constexpr int kMaxL = 1024;

struct SearchArgs {
    const void *queries;      // device, nq*d elements
    const float *codebook;    // device, 256*d
    const uint32_t *off;      // device, M+1
    const uint8_t *codes;     // device, n*Mpad
    const uint32_t *adj;      // device-accessible (mapped host), n*R
    const void *base;         // device-accessible (mapped host), n*d
    uint32_t n, d, M, Mpad, R, medoid;
    uint32_t nq, k, L, log2z, iter_cap;
    uint32_t *out_ids;        // device, nq*k
    float *out_dist;          // device, nq*k
    uint32_t *out_iters;      // device or null
    int32_t *out_status;      // device or null
    uint32_t *out_ndist;      // device or null
    uint32_t *trace;          // device or null
    uint32_t trace_cap;
};

// Shared-memory carve-up, in bytes, shared by host (sizing) and device.
struct SmemLayout {
    uint32_t off_T, off_bloom, off_L0, off_L1, off_Nk, off_Nid, off_cnt, off_Ck, off_q, off_offs,
        total;
    __host__ __device__ static uint32_t up16(uint32_t x) { return (x + 15u) & ~15u; }
    __host__ __device__ SmemLayout(uint32_t M, uint32_t log2z, uint32_t L, uint32_t k, uint32_t d)
    {
        uint32_t o = 0;
        off_T = o;      o += up16(M * 256u * 4u);
        off_bloom = o;  o += up16(((1u << log2z) / 8u) < 4u ? 4u : (1u << log2z) / 8u);
        off_L0 = o;     o += up16(L * 8u);
        off_L1 = o;     o += up16(L * 8u);
        off_Nk = o;     o += up16(kMaxR * 8u);
        off_Nid = o;    o += up16(kMaxR * 4u);
        off_cnt = o;    o += up16((L + 1u) * 4u);
        off_Ck = o;     o += up16(k * 8u);
        off_q = o;      o += up16(d * 4u);
        off_offs = o;   o += up16((M + 1u) * 4u);
        total = o;
    }
};

template <int DT> struct Elem;
template <> struct Elem<0> { using T = uint8_t; };
template <> struct Elem<1> { using T = int8_t; };
template <> struct Elem<2> { using T = float; };

__device__ __forceinline__ uint64_t make_key(uint32_t dbits, uint32_t id)
{
    return (static_cast<uint64_t>(dbits) << 32) | (static_cast<uint64_t>(id) << 1);
}
__device__ __forceinline__ uint32_t key_id(uint64_t key) { return static_cast<uint32_t>(key) >> 1; }

// FNV-1a over the four little-endian bytes of the id (32-bit, and 64-bit
// folded to 32 bits), the two hash functions of the per-query Bloom filter.
__device__ __forceinline__ uint32_t fnv1a32_id(uint32_t id)
{
    uint32_t h = 2166136261u;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        h ^= (id >> (8 * b)) & 0xFFu;
        h *= 16777619u;
    }
    return h;
}
__device__ __forceinline__ uint32_t fnv1a64_id_folded(uint32_t id)
{
    uint64_t h = 14695981039346656037ull;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        h ^= static_cast<uint64_t>((id >> (8 * b)) & 0xFFu);
        h *= 1099511628211ull;
    }
    return static_cast<uint32_t>(h >> 32) ^ static_cast<uint32_t>(h);
}

__device__ __forceinline__ uint64_t shfl_xor_u64(uint64_t v, int m)
{
    uint32_t lo = __shfl_xor_sync(0xFFFFFFFFu, static_cast<uint32_t>(v), m);
    uint32_t hi = __shfl_xor_sync(0xFFFFFFFFu, static_cast<uint32_t>(v >> 32), m);
    return (static_cast<uint64_t>(hi) << 32) | lo;
}
__device__ __forceinline__ uint64_t warp_min_u64(uint64_t v)
{
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) {
        uint64_t o = shfl_xor_u64(v, m);
        v = o < v ? o : v;
    }
    return v;
}
__device__ __forceinline__ uint32_t warp_sum_u32(uint32_t v)
{
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, m);
    return v;
}

// PQ distance of one code row (§4.4), in the fixed order described above.
__device__ __forceinline__ float adc_distance(const float *__restrict__ T,
                                              const uint8_t *__restrict__ row, uint32_t M,
                                              uint32_t Mpad)
{
    float p[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) p[r] = 0.0f;
    const uint4 *row16 = reinterpret_cast<const uint4 *>(row);
    for (uint32_t c16 = 0; c16 < Mpad / 16u; ++c16) {
        uint4 v = __ldg(row16 + c16);
        uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int b = 0; b < 16; ++b) {
            uint32_t s = c16 * 16u + static_cast<uint32_t>(b);
            uint32_t code = (w[b >> 2] >> (8 * (b & 3))) & 0xFFu;
            if (s < M) p[b & 7] = __fadd_rn(p[b & 7], T[s * 256u + code]);
        }
    }
#pragma unroll
    for (int h = 4; h >= 1; h >>= 1) {
        float nx[8];
#pragma unroll
        for (int r = 0; r < 8; ++r) nx[r] = __fadd_rn(p[r], p[r ^ h]);
#pragma unroll
        for (int r = 0; r < 8; ++r) p[r] = nx[r];
    }
    return p[0];
}

// The expanded node's neighbour ids and this lane's share of its vector.
template <int DT> struct NodeData {
    uint32_t nb[kMaxRPL];
    float xf[kMaxDPL];
    int32_t xi[kMaxDPL];
};

template <int DT>
__device__ __forceinline__ void load_node(const SearchArgs &a, uint32_t u, int lane,
                                          NodeData<DT> &nd)
{
    using E = typename Elem<DT>::T;
    const uint32_t *row = a.adj + static_cast<uint64_t>(u) * a.R;
#pragma unroll
    for (int r = 0; r < kMaxRPL; ++r) {
        uint32_t i = static_cast<uint32_t>(lane + kWarp * r);
        nd.nb[r] = i < a.R ? row[i] : kNone;
    }
    const E *x = static_cast<const E *>(a.base) + static_cast<uint64_t>(u) * a.d;
#pragma unroll
    for (int t = 0; t < kMaxDPL / 4; ++t) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            uint32_t j = 128u * t + 4u * lane + i;
            if (DT == 2) nd.xf[4 * t + i] = j < a.d ? static_cast<float>(x[j]) : 0.0f;
            else nd.xi[4 * t + i] = j < a.d ? static_cast<int32_t>(x[j]) : 0;
        }
    }
}

template <int DT>
__global__ void __launch_bounds__(32) search_kernel(const SearchArgs a)
{
    using E = typename Elem<DT>::T;
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x;
    const SmemLayout lay(a.M, a.log2z, a.L, a.k, a.d);
    float *T = reinterpret_cast<float *>(smem + lay.off_T);
    uint32_t *bloom = reinterpret_cast<uint32_t *>(smem + lay.off_bloom);
    uint64_t *Lbuf0 = reinterpret_cast<uint64_t *>(smem + lay.off_L0);
    uint64_t *Lbuf1 = reinterpret_cast<uint64_t *>(smem + lay.off_L1);
    uint64_t *Nk = reinterpret_cast<uint64_t *>(smem + lay.off_Nk);
    uint32_t *Nid = reinterpret_cast<uint32_t *>(smem + lay.off_Nid);
    uint32_t *cnt = reinterpret_cast<uint32_t *>(smem + lay.off_cnt);
    uint64_t *Ck = reinterpret_cast<uint64_t *>(smem + lay.off_Ck);
    float *qv = reinterpret_cast<float *>(smem + lay.off_q);
    uint32_t *offs = reinterpret_cast<uint32_t *>(smem + lay.off_offs);

    const uint32_t M = a.M, d = a.d, L = a.L, k = a.k;
    const uint32_t zmask = (1u << a.log2z) - 1u;
    const uint32_t nwords = (1u << a.log2z) >= 32u ? (1u << a.log2z) / 32u : 1u;

    for (uint32_t i = lane; i <= M; i += kWarp) offs[i] = a.off[i];

    for (uint32_t q = blockIdx.x; q < a.nq; q += gridDim.x) {
        // ---- query: FP32 copy in shared memory, this lane's share in registers
        const E *qp = static_cast<const E *>(a.queries) + static_cast<uint64_t>(q) * d;
        for (uint32_t j = lane; j < d; j += kWarp) qv[j] = static_cast<float>(qp[j]);
        float qf[kMaxDPL];
        int32_t qi[kMaxDPL];
#pragma unroll
        for (int t = 0; t < kMaxDPL / 4; ++t)
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                uint32_t j = 128u * t + 4u * lane + i;
                qf[4 * t + i] = j < d ? static_cast<float>(qp[j]) : 0.0f;
                qi[4 * t + i] = j < d ? static_cast<int32_t>(qp[j]) : 0;
            }
        for (uint32_t w = lane; w < nwords; w += kWarp) bloom[w] = 0u;
        __syncwarp();

        // ---- PQ distance table, §4.1
        for (uint32_t idx = lane; idx < M * 256u; idx += kWarp) {
            uint32_t s = idx >> 8, c = idx & 255u;
            uint32_t o = offs[s], ds = offs[s + 1] - o;
            const float *cc = a.codebook + 256u * o + c * ds;
            float acc = 0.0f;
            for (uint32_t j = 0; j < ds; ++j) {
                float df = __fsub_rn(qv[o + j], __ldg(cc + j));
                acc = __fmaf_rn(df, df, acc);
            }
            T[idx] = acc;
        }
        __syncwarp();

        // ---- start: worklist = {medoid}, medoid marked seen
        uint64_t *Lcur = Lbuf0, *Lnext = Lbuf1;
        if (lane == 0) {
            uint32_t s = a.medoid;
            float dm = adc_distance(T, a.codes + static_cast<uint64_t>(s) * a.Mpad, M, a.Mpad);
            Lcur[0] = make_key(__float_as_uint(dm), s);
            uint32_t p1 = fnv1a32_id(s) & zmask, p2 = fnv1a64_id_folded(s) & zmask;
            bloom[p1 >> 5] |= 1u << (p1 & 31u);
            bloom[p2 >> 5] |= 1u << (p2 & 31u);
        }
        uint32_t nl = 1, nc = 0, iters = 0, ndist = 1;
        int32_t status = 0;
        uint32_t cur = a.medoid;
        NodeData<DT> nd;
        load_node<DT>(a, cur, lane, nd);
        __syncwarp();

        for (;;) {
            // u* = first unvisited entry of the sorted worklist (Alg. 1)
            int first = -1;
            for (uint32_t b0 = 0; b0 < nl; b0 += kWarp) {
                uint32_t i = b0 + lane;
                bool v = i < nl && !(Lcur[i] & 1ull);
                uint32_t bal = __ballot_sync(0xFFFFFFFFu, v);
                if (bal) {
                    first = static_cast<int>(b0 + __ffs(bal) - 1);
                    break;
                }
            }
            if (first < 0) break;
            if (iters >= a.iter_cap) {
                status = 1;
                break;
            }
            const uint64_t ukey = Lcur[first];
            const uint32_t u = key_id(ukey);
            __syncwarp();
            if (lane == 0) {
                Lcur[first] = ukey | 1ull;
                if (a.trace && iters < a.trace_cap)
                    a.trace[static_cast<uint64_t>(q) * a.trace_cap + iters] = u;
            }
            ++iters;
            if (u != cur) {  // the prefetched node is always u*; reload if not
                cur = u;
                load_node<DT>(a, cur, lane, nd);
            }

            // ---- re-rank candidate: exact distance of u* (§4.8)
            uint32_t ebits;
            if (DT == 2) {
                float p = 0.0f;
#pragma unroll
                for (int t = 0; t < kMaxDPL; ++t) {
                    float df = __fsub_rn(qf[t], nd.xf[t]);
                    p = __fmaf_rn(df, df, p);
                }
#pragma unroll
                for (int m = 16; m >= 1; m >>= 1) p = __fadd_rn(p, __shfl_xor_sync(0xFFFFFFFFu, p, m));
                ebits = __float_as_uint(p);
            } else {
                int32_t p = 0;
#pragma unroll
                for (int t = 0; t < kMaxDPL; ++t) {
                    int32_t df = qi[t] - nd.xi[t];
                    p += df * df;
                }
                ebits = warp_sum_u32(static_cast<uint32_t>(p));
            }
            {
                const uint64_t e = make_key(ebits, u);
                if (!(nc == k && e >= Ck[k - 1])) {
                    uint32_t less = 0;
                    uint64_t keep[kMaxK / kWarp];
#pragma unroll
                    for (int t = 0; t < kMaxK / kWarp; ++t) {
                        uint32_t i = lane + kWarp * t;
                        keep[t] = i < nc ? Ck[i] : 0ull;
                        less += (i < nc && keep[t] < e) ? 1u : 0u;
                    }
                    const uint32_t pos = warp_sum_u32(less);
                    __syncwarp();
#pragma unroll
                    for (int t = 0; t < kMaxK / kWarp; ++t) {
                        uint32_t i = lane + kWarp * t;
                        if (i < nc && i >= pos && i + 1 < k) Ck[i + 1] = keep[t];
                    }
                    if (lane == 0) Ck[pos] = e;
                    nc = nc + 1 < k ? nc + 1 : k;
                    __syncwarp();
                }
            }

            // ---- filter seen neighbours, §4.3: test all, then insert all
            bool fresh[kMaxRPL];
            uint32_t p1[kMaxRPL], p2[kMaxRPL];
#pragma unroll
            for (int r = 0; r < kMaxRPL; ++r) {
                uint32_t id = nd.nb[r];
                fresh[r] = false;
                if (id != kNone) {
                    p1[r] = fnv1a32_id(id) & zmask;
                    p2[r] = fnv1a64_id_folded(id) & zmask;
                    bool hit = ((bloom[p1[r] >> 5] >> (p1[r] & 31u)) & 1u) &&
                               ((bloom[p2[r] >> 5] >> (p2[r] & 31u)) & 1u);
                    fresh[r] = !hit;
                }
            }
            __syncwarp();
            uint32_t nn = 0;
#pragma unroll
            for (int r = 0; r < kMaxRPL; ++r) {
                if (fresh[r]) {
                    atomicOr(&bloom[p1[r] >> 5], 1u << (p1[r] & 31u));
                    atomicOr(&bloom[p2[r] >> 5], 1u << (p2[r] & 31u));
                }
                uint32_t bal = __ballot_sync(0xFFFFFFFFu, fresh[r]);
                if (fresh[r]) Nid[nn + __popc(bal & ((1u << lane) - 1u))] = nd.nb[r];
                nn += __popc(bal);
            }
            __syncwarp();

            // ---- PQ distances of the new neighbours, §4.4
            for (uint32_t j = lane; j < nn; j += kWarp) {
                uint32_t id = Nid[j];
                float dj = adc_distance(T, a.codes + static_cast<uint64_t>(id) * a.Mpad, M, a.Mpad);
                Nk[j] = make_key(__float_as_uint(dj), id);
            }
            ndist += nn;
            __syncwarp();

            // ---- eager next node, §4.5: best of the new neighbours and the
            // first unvisited worklist entry after u*; prefetch its lists
            {
                uint64_t best = ~0ull;
                for (uint32_t j = lane; j < nn; j += kWarp) best = Nk[j] < best ? Nk[j] : best;
                for (uint32_t b0 = static_cast<uint32_t>(first) + 1; b0 < nl; b0 += kWarp) {
                    uint32_t i = b0 + lane;
                    bool v = i < nl && !(Lcur[i] & 1ull);
                    uint32_t bal = __ballot_sync(0xFFFFFFFFu, v);
                    if (bal) {
                        uint32_t f = b0 + __ffs(bal) - 1;
                        uint64_t lk = Lcur[f];
                        best = lk < best ? lk : best;
                        break;
                    }
                }
                best = warp_min_u64(best);
                if (best != ~0ull) {
                    cur = key_id(best);
                    load_node<DT>(a, cur, lane, nd);
                }
            }

            // ---- merge the new neighbours into the worklist, §4.6-§4.7:
            // every element's output position is its index plus its rank in
            // the other list; keys are unique, so ranks are exact
            for (uint32_t i = lane; i <= nl; i += kWarp) cnt[i] = 0u;
            __syncwarp();
            for (uint32_t j = lane; j < nn; j += kWarp) {
                const uint64_t x = Nk[j];
                uint32_t lo = 0, hi = nl;          // rank in the worklist
                while (lo < hi) {
                    uint32_t mid = (lo + hi) >> 1;
                    if ((Lcur[mid] >> 1) < (x >> 1)) lo = mid + 1;
                    else hi = mid;
                }
                uint32_t rn = 0;                   // rank among the new ones
                for (uint32_t t = 0; t < nn; ++t) rn += Nk[t] < x ? 1u : 0u;
                const uint32_t pos = lo + rn;
                if (pos < L) Lnext[pos] = x;
                atomicAdd(&cnt[lo], 1u);
            }
            __syncwarp();
            {
                uint32_t carry = 0;
                for (uint32_t b0 = 0; b0 < nl; b0 += kWarp) {
                    uint32_t i = b0 + lane;
                    uint32_t v = i < nl ? cnt[i] : 0u;
#pragma unroll
                    for (int m = 1; m < kWarp; m <<= 1) {
                        uint32_t o = __shfl_up_sync(0xFFFFFFFFu, v, m);
                        if (lane >= m) v += o;
                    }
                    v += carry;
                    if (i < nl) {
                        uint32_t pos = i + v;
                        if (pos < L) Lnext[pos] = Lcur[i];
                    }
                    carry = __shfl_sync(0xFFFFFFFFu, v, kWarp - 1);
                }
            }
            nl = nl + nn < L ? nl + nn : L;
            uint64_t *tmp = Lcur;
            Lcur = Lnext;
            Lnext = tmp;
            __syncwarp();
        }

        // ---- output: re-ranked top-k (§4.8), padded
        for (uint32_t i = lane; i < k; i += kWarp) {
            uint64_t o = static_cast<uint64_t>(q) * k + i;
            if (i < nc) {
                uint64_t key = Ck[i];
                uint32_t bits = static_cast<uint32_t>(key >> 32);
                a.out_ids[o] = key_id(key);
                a.out_dist[o] = DT == 2 ? __uint_as_float(bits) : static_cast<float>(bits);
            } else {
                a.out_ids[o] = kNone;
                a.out_dist[o] = __uint_as_float(0x7F800000u);
            }
        }
        if (lane == 0) {
            if (a.out_iters) a.out_iters[q] = iters;
            if (a.out_status) a.out_status[q] = status;
            if (a.out_ndist) a.out_ndist[q] = ndist;
        }
        __syncwarp();
    }
}

}  // namespace bang
