// Greedy-search kernel of BANG (arXiv 2401.11324), FP32 form, for sm_103a.
//
// One warp (a 32-thread CTA) runs the whole search of one query: the PQ
// distance table (§4.1), the Bloom-filter seen set (§4.3), the worklist and
// the re-rank's running top-k all live in shared memory or registers, so the
// only global traffic per iteration is the neighbour row and full vector of
// the expanded node (read in place from page-locked host memory, Alg. 2
// "FetchNeighbors", or from HBM) and one PQ code row per new neighbour (HBM,
// §4.4).  With the staged re-rank the loop records the expanded nodes
// instead and fetches no vectors; rerank.cu ranks them afterwards (§4.8).
//
// The paper splits every iteration into separate kernels with one CTA per
// query and keeps the table and filter in global memory; here the iteration
// loop stays inside one warp, and the eager next-node choice of §4.5 becomes
// a software prefetch: the next node's lists are requested right after the
// distances are known and arrive while the warp merges the worklist.
//
// Arithmetic order (fixed so that results are reproducible bit for bit):
//  - table entry T[s][c]: fmaf(q_j - C_j, q_j - C_j, acc) over the subspace's
//    dimensions in ascending j, from 0;
//  - PQ distance: eight partial sums over subspaces s = r (mod 8), in
//    ascending s, then p_r += p_(r^4), p_r += p_(r^2), p_r += p_(r^1);
//    on the 8-bit table an exact integer sum;
//  - exact distance: 32 partial sums, lane r owning the dimensions j with
//    (j/4) mod 32 = r, each in ascending j (fmaf), then a butterfly over xor
//    distances 16, 8, 4, 2, 1; integer data is summed exactly;
//  - ordering keys are (distance, id): FP32 distances compared through their
//    bit patterns (all distances are >= +0), integer exact distances as
//    unsigned integers.
#pragma once

#include <atomic>
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace bang {

constexpr uint32_t kNone = 0xFFFFFFFFu;
constexpr int kWarp = 32;
constexpr int kMaxR = 128;        // neighbours per row: up to 4 per lane
constexpr int kMaxD = 512;        // dimensions: up to 16 per lane for the exact distance
constexpr int kMaxM = 128;
constexpr int kMaxK = 256;
constexpr int kMaxL = 1024;
constexpr int kRegK = 32;         // k up to this keeps the re-rank top-k in registers

// Distance modes of the search loop.
//  kModeF32:   PQ distances from an FP32 table (the bit-exact form, §4.1, §4.4)
//  kModeBF16:  PQ distances from a BF16 table, summed in FP32 (reduced form:
//              half the table's shared memory, so more queries per SM)
//  kModeExact: exact distances to the full vectors in the loop, no table and
//              no re-rank (the paper's Exact-distance variant, §5.2)
//  kModeQ8:    PQ distances from an 8-bit table (per-subspace offset, one
//              scale per query) summed exactly in integers: a quarter of the
//              FP32 table's shared memory; not in the paper
//  kModeF32Lazy: the FP32 form with a partial table or none: the first ntab
//              subspaces' entries are kept in shared memory, every other
//              entry a distance needs is computed from the query and the
//              codebook (read through L1) in the table's own arithmetic, so
//              the sums are kModeF32's bit for bit while a query holds less
//              than the 32 KB table and more queries fit on an SM
enum { kModeF32 = 0, kModeBF16 = 1, kModeExact = 2, kModeQ8 = 3, kModeF32Lazy = 4 };

struct SearchArgs {
    const void *queries;      // device, nq*d elements
    const float *codebook;    // device, 256*d
    const uint32_t *off;      // device, M+1
    const uint8_t *codes;     // device, n*Mpad
    const uint32_t *adj;      // device-accessible (mapped host), n rows of adj_row_words words
    uint32_t adj_bits;        // 0: rows of R ids; else ids packed to adj_bits bits, all ones = none
    uint32_t adj_row_words;   // 32-bit words per row (R when not packed)
    uint32_t adj_stride;      // 32-bit words from one row to the next (>= the row's words)
    const uint8_t *ncodes;    // device or null: for every node, its R neighbours' code rows, 32 bytes each
    uint32_t spec;            // also request the first unvisited worklist entry after u* at once
    const void *base;         // device-accessible (mapped host), n vectors of d elements
    uint32_t vstride;         // elements from one vector to the next (>= d)
    uint32_t n, d, M, Mpad, R, medoid;
    uint32_t nq, k, L, log2z, iter_cap;
    uint32_t vec_ok;          // rows of `queries` allow 4-element vector loads
    uint32_t vecb_ok;         // rows of `base` allow 4-element vector loads
    uint32_t *out_ids;        // device, nq*k
    float *out_dist;          // device, nq*k
    uint32_t *out_iters;      // device or null
    int32_t *out_status;      // device or null
    uint32_t *out_ndist;      // device or null
    uint32_t *trace;          // device or null
    uint32_t trace_cap;
    // Batched form: per-query k and L (device or null: every query uses k, L,
    // which are otherwise the bounds and the output row stride), an optional
    // processing order and a work counter for the persistent launch.
    const uint32_t *k_per_q;
    const uint32_t *L_per_q;
    const uint32_t *order;
    unsigned int *queue;      // device counter, zero at launch; null: grid covers the queries
    uint32_t grid_mult;       // persistent grid = grid_mult x resident CTAs (>= 1)
    const void *tables;       // BF16 or FP32 mode: nq*M*256 precomputed tables (tensor cores), or null
    const unsigned int *tables_err;  // set when the table kernel gave up
    unsigned long long *phase_cycles;  // device or null: nq*kPhases SM cycles per phase
    const uint32_t *entry;    // device or null: per-query start node (null: every query starts at medoid)
    uint32_t early_codes;     // request every neighbour's code row as soon as the row arrives (see CS)
    // Staged re-rank (PQ modes): when `cand` is set the loop fetches no
    // vectors and keeps no top-k; it records every expanded node, the
    // candidate set of §4.8, in row q of `cand` (cand_cap >= the iteration
    // cap, so no candidate is lost), or with cand_list the final worklist,
    // and their number in cand_n[q]; the re-rank kernel computes the exact
    // distances and the top-k afterwards.
    uint32_t *cand;
    uint32_t cand_cap;
    uint32_t *cand_n;
    uint32_t cand_list;       // 1: the candidates are the final worklist instead (cand_cap >= L)
    uint32_t carveout;        // preferred shared-memory share of L1 in percent (0: the CUDA driver's choice)
    uint32_t ntab;            // kModeF32Lazy: subspaces (the first ones) whose entries stay in a table
};

// Phases timed when SearchArgs::phase_cycles is set.
enum Phase { kPhTable = 0, kPhSelect, kPhFilter, kPhDistance, kPhNext, kPhRerank, kPhMerge,
             kPhMergeRank, kPhMergeShift, kPhTotal, kPhases };

// Shared-memory carve-up, in bytes, shared by host (sizing) and device.
struct SmemLayout {
    uint32_t off_T, off_bloom, off_L, off_Nk, off_Nid, off_Ck, off_q, off_offs, off_lo, total;
    __host__ __device__ static uint32_t up16(uint32_t x) { return (x + 15u) & ~15u; }
    // ntab: kModeF32Lazy only, the subspaces whose FP32 entries are kept
    __host__ __device__ SmemLayout(uint32_t M, uint32_t log2z, uint32_t L, uint32_t k, uint32_t d,
                                   uint32_t R, int mode, uint32_t ntab = 0)
    {
        uint32_t o = 0;
        const bool lazy = mode == kModeF32Lazy;       // query and offsets stay live in the loop
        const uint32_t tsz = mode == kModeF32 || lazy ? 4u : mode == kModeBF16 ? 2u : mode == kModeQ8 ? 1u : 0u;
        const uint32_t tsub = lazy ? (ntab < M ? ntab : M) : M;
        const uint32_t rw = (R + 31u) & ~31u;          // neighbour slots: whole lanes' worth
        off_T = o;      o += up16(tsub * 256u * tsz);
        off_bloom = o;  o += up16(((1u << log2z) / 8u) < 4u ? 4u : (1u << log2z) / 8u);
        off_L = o;      o += up16(L * 8u);
        off_Nk = o;     o += up16(rw * 8u);
        off_Nid = o;    o += up16(rw * 4u);
        off_Ck = o;     o += up16(k > (uint32_t)kRegK && mode != kModeExact ? k * 8u : 0u);
        // table-build scratch (query, subspace offsets, 8-bit-table minima):
        // dead once the table is built, so it shares the worklist's space
        // when that is large enough (not without a table: the loop reads it)
        const uint32_t sq = up16(mode != kModeExact ? d * 4u : 0u), so = up16((M + 1u) * 4u),
                       sl = up16(mode == kModeQ8 ? M * 4u : 0u);
        uint32_t b = !lazy && up16(L * 8u) >= sq + so + sl ? off_L : o;
        off_q = b;      b += sq;
        off_offs = b;   b += so;
        off_lo = b;     b += sl;
        if (off_q != off_L) o = b;
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
// folded to 32 bits): the two hash functions of the per-query Bloom filter.
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

// Minimum of a 64-bit key over the warp: high words first, then the low
// words of the lanes that hold the minimal high word.
__device__ __forceinline__ uint64_t warp_min_key(uint64_t v)
{
    uint32_t hi = __reduce_min_sync(0xFFFFFFFFu, static_cast<uint32_t>(v >> 32));
    uint32_t lo = __reduce_min_sync(0xFFFFFFFFu, static_cast<uint32_t>(v >> 32) == hi
                                                     ? static_cast<uint32_t>(v) : 0xFFFFFFFFu);
    return (static_cast<uint64_t>(hi) << 32) | lo;
}

__device__ __forceinline__ uint64_t shfl_u64(uint64_t v, int src)
{
    uint32_t lo = __shfl_sync(0xFFFFFFFFu, static_cast<uint32_t>(v), src);
    uint32_t hi = __shfl_sync(0xFFFFFFFFu, static_cast<uint32_t>(v >> 32), src);
    return (static_cast<uint64_t>(hi) << 32) | lo;
}
__device__ __forceinline__ uint64_t shfl_up_u64(uint64_t v, int delta)
{
    uint32_t lo = __shfl_up_sync(0xFFFFFFFFu, static_cast<uint32_t>(v), delta);
    uint32_t hi = __shfl_up_sync(0xFFFFFFFFu, static_cast<uint32_t>(v >> 32), delta);
    return (static_cast<uint64_t>(hi) << 32) | lo;
}

// Where a query's table entries come from: its table in shared memory, or,
// without a table (kModeF32Lazy), the query, the subspace offsets and the
// codebook, from which an entry is computed when a distance needs it.
struct TableRef {
    const void *T;              // the table (modes with one)
    const float *qv;            // the query in FP32 (shared memory)
    const uint32_t *offs;       // subspace offsets, M + 1 (shared memory)
    const float *codebook;      // 256 centroids per subspace, subspace-major (global)
    uint32_t ds;                // dimensions per subspace when all are equal, else 0
    uint32_t ntab;              // kModeF32Lazy: subspaces s < ntab read from T (FP32)
};

// Table entry T[s][c] as FP32: FP32 tables are read directly, BF16 entries
// widened; without a table the entry is computed in the table build's
// arithmetic (fmaf of the differences in ascending j, from 0), so it has
// the bits the FP32 table would hold.
template <int MODE> __device__ __forceinline__ float table_entry(const TableRef &t, uint32_t s, uint32_t c)
{
    if constexpr (MODE == kModeBF16) {
        return __uint_as_float(static_cast<uint32_t>(static_cast<const uint16_t *>(t.T)[s * 256u + c]) << 16);
    } else if constexpr (MODE == kModeF32Lazy) {
        if (s < t.ntab) return static_cast<const float *>(t.T)[s * 256u + c];
        uint32_t o, ds;
        if (t.ds) {
            ds = t.ds;
            o = s * ds;
        } else {
            o = t.offs[s];
            ds = t.offs[s + 1] - o;
        }
        const float *cc = t.codebook + 256u * o + c * ds;
        float acc = 0.0f, df;
        if (ds == 4 && (o & 3u) == 0) {
            const float4 q4 = *reinterpret_cast<const float4 *>(t.qv + o);
            const float4 c4 = __ldg(reinterpret_cast<const float4 *>(cc));
            df = __fsub_rn(q4.x, c4.x); acc = __fmaf_rn(df, df, acc);
            df = __fsub_rn(q4.y, c4.y); acc = __fmaf_rn(df, df, acc);
            df = __fsub_rn(q4.z, c4.z); acc = __fmaf_rn(df, df, acc);
            df = __fsub_rn(q4.w, c4.w); acc = __fmaf_rn(df, df, acc);
        } else {
            for (uint32_t j = 0; j < ds; ++j) {
                df = __fsub_rn(t.qv[o + j], __ldg(cc + j));
                acc = __fmaf_rn(df, df, acc);
            }
        }
        return acc;
    } else {
        return static_cast<const float *>(t.T)[s * 256u + c];
    }
}

// PQ distance of one code row on the 8-bit table: the exact integer sum of
// the selected entries (any order gives the same sum).
// `get(c16)` returns the code row's 16-byte chunk c16 (from memory, or from
// registers loaded earlier).
template <typename Get>
__device__ __forceinline__ uint32_t adc_distance_q8(const uint8_t *__restrict__ T, Get get, uint32_t M,
                                                    uint32_t Mpad)
{
    uint32_t p[4] = {0u, 0u, 0u, 0u};
    for (uint32_t c16 = 0; c16 < Mpad / 16u; ++c16) {
        uint4 v = get(c16);
        uint32_t w[4] = {v.x, v.y, v.z, v.w};
        const uint8_t *tc = T + c16 * 16u * 256u;
        if (c16 * 16u + 16u <= M) {
#pragma unroll
            for (int b = 0; b < 16; ++b) p[b & 3] += tc[b * 256 + ((w[b >> 2] >> (8 * (b & 3))) & 0xFFu)];
        } else {
#pragma unroll
            for (int b = 0; b < 16; ++b)
                if (c16 * 16u + b < M) p[b & 3] += tc[b * 256 + ((w[b >> 2] >> (8 * (b & 3))) & 0xFFu)];
        }
    }
    return (p[0] + p[1]) + (p[2] + p[3]);
}

// PQ distance of one code row (§4.4), in the fixed order described above.
template <int MODE, typename Get>
__device__ __forceinline__ float adc_distance(const TableRef &t, Get get, uint32_t M, uint32_t Mpad)
{
    float p[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) p[r] = 0.0f;
    for (uint32_t c16 = 0; c16 < Mpad / 16u; ++c16) {
        uint4 v = get(c16);
        uint32_t w[4] = {v.x, v.y, v.z, v.w};
        const uint32_t s0 = c16 * 16u;
        if (s0 + 16u <= M) {
#pragma unroll
            for (int b = 0; b < 16; ++b)
                p[b & 7] = __fadd_rn(p[b & 7], table_entry<MODE>(t, s0 + b, (w[b >> 2] >> (8 * (b & 3))) & 0xFFu));
        } else {
#pragma unroll
            for (int b = 0; b < 16; ++b)
                if (s0 + b < M)
                    p[b & 7] = __fadd_rn(p[b & 7], table_entry<MODE>(t, s0 + b, (w[b >> 2] >> (8 * (b & 3))) & 0xFFu));
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

// This lane's share of a vector for the exact distance: dimensions
// 128*t + 4*lane + i, i < 4, t < DCH.  Integer data is packed four bytes per
// word (int8 biased by 0x80 so that byte differences are unsigned).
// Ordering bits of a PQ distance: FP32 distances (all >= +0) through their
// bit patterns, 8-bit-table sums as integers.
template <int MODE, typename Get>
__device__ __forceinline__ uint32_t pq_dist_bits_g(const TableRef &t, Get get, uint32_t M, uint32_t Mpad)
{
    if constexpr (MODE == kModeQ8)
        return adc_distance_q8(static_cast<const uint8_t *>(t.T), get, M, Mpad);
    else
        return __float_as_uint(adc_distance<MODE>(t, get, M, Mpad));
}

template <int MODE>
__device__ __forceinline__ uint32_t pq_dist_bits(const TableRef &t, const uint8_t *row, uint32_t M,
                                                 uint32_t Mpad)
{
    const uint4 *row16 = reinterpret_cast<const uint4 *>(row);
    return pq_dist_bits_g<MODE>(t, [row16](uint32_t c16) { return __ldg(row16 + c16); }, M, Mpad);
}

// Part of an 8-bit-table PQ distance: the 8-byte chunks c = part, part + P,
// ... of the code row (rows are padded to 16 bytes).  P lanes together give
// the exact integer sum of the whole row.
template <uint32_t P>
__device__ __forceinline__ uint32_t adc_q8_part(const uint8_t *__restrict__ T, const uint8_t *row, uint32_t M,
                                                uint32_t Mpad, uint32_t part)
{
    uint32_t p[4] = {0u, 0u, 0u, 0u};
    const uint2 *row8 = reinterpret_cast<const uint2 *>(row);
    for (uint32_t c = part; c < Mpad / 8u; c += P) {
        const uint2 v = __ldg(row8 + c);
        const uint32_t w[2] = {v.x, v.y};
        const uint8_t *tc = T + c * 8u * 256u;
        if (c * 8u + 8u <= M) {
#pragma unroll
            for (int b = 0; b < 8; ++b) p[b & 3] += tc[b * 256 + ((w[b >> 2] >> (8 * (b & 3))) & 0xFFu)];
        } else {
#pragma unroll
            for (int b = 0; b < 8; ++b)
                if (c * 8u + b < M) p[b & 3] += tc[b * 256 + ((w[b >> 2] >> (8 * (b & 3))) & 0xFFu)];
        }
    }
    return (p[0] + p[1]) + (p[2] + p[3]);
}

// 8-bit-table PQ distances of up to 32 / P new neighbours, P lanes each:
// neighbour j = lane / P, its key left in lane P*j (kv set there only).
template <uint32_t P>
__device__ __forceinline__ void pq_q8_split(const SearchArgs &a, const uint8_t *T, const uint32_t *Nid,
                                            uint32_t nn, int lane, uint64_t &kk, bool &kv)
{
    const uint32_t j = static_cast<uint32_t>(lane) / P, part = static_cast<uint32_t>(lane) % P;
    const bool act = j < nn;
    const uint32_t id = act ? Nid[j] : 0u;
    uint32_t s = act ? adc_q8_part<P>(T, a.codes + static_cast<uint64_t>(id) * a.Mpad, a.M, a.Mpad, part) : 0u;
#pragma unroll
    for (uint32_t h = 1; h < P; h <<= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, static_cast<int>(h));
    kv = act && part == 0u;
    kk = kv ? make_key(s, id) : ~0ull;
}

template <int DT, int DCH> struct VecShare {
    float f[DT == 2 ? 4 * DCH : 1];
    uint32_t w[DT == 2 ? 1 : DCH];
};

template <int DT, int DCH>
__device__ __forceinline__ void load_share(const typename Elem<DT>::T *x, uint32_t d, bool vec,
                                           int lane, VecShare<DT, DCH> &v)
{
#pragma unroll
    for (int t = 0; t < DCH; ++t) {
        const uint32_t j0 = 128u * t + 4u * lane;
        if (DT == 2) {
            if (vec) {
                float4 f4 = j0 < d ? *reinterpret_cast<const float4 *>(x + j0)
                                   : make_float4(0.f, 0.f, 0.f, 0.f);
                v.f[4 * t + 0] = f4.x; v.f[4 * t + 1] = f4.y;
                v.f[4 * t + 2] = f4.z; v.f[4 * t + 3] = f4.w;
            } else {
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    v.f[4 * t + i] = (j0 + i < d) ? static_cast<float>(x[j0 + i]) : 0.0f;
            }
        } else {
            uint32_t w = 0;
            if (vec) {
                w = j0 < d ? *reinterpret_cast<const uint32_t *>(x + j0) : 0u;
            } else {
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    if (j0 + i < d) w |= static_cast<uint32_t>(static_cast<uint8_t>(x[j0 + i])) << (8 * i);
            }
            if (DT == 1) {
                // bias only the dimensions that exist, so padding stays equal on both sides
                uint32_t m = 0;
#pragma unroll
                for (int i = 0; i < 4; ++i) if (j0 + i < d) m |= 0x80u << (8 * i);
                w ^= m;
            }
            v.w[t] = w;
        }
    }
}

template <int DT, int DCH>
__device__ __forceinline__ uint32_t exact_distance_bits(const VecShare<DT, DCH> &q,
                                                        const VecShare<DT, DCH> &x)
{
    if (DT == 2) {
        float p = 0.0f;
#pragma unroll
        for (int t = 0; t < 4 * DCH; ++t) {
            float df = __fsub_rn(q.f[t], x.f[t]);
            p = __fmaf_rn(df, df, p);
        }
#pragma unroll
        for (int m = 16; m >= 1; m >>= 1) p = __fadd_rn(p, __shfl_xor_sync(0xFFFFFFFFu, p, m));
        return __float_as_uint(p);
    } else {
        uint32_t acc = 0;
#pragma unroll
        for (int t = 0; t < DCH; ++t) {
            uint32_t df = __vabsdiffu4(q.w[t], x.w[t]);
            acc = __dp4a(df, df, acc);
        }
        return __reduce_add_sync(0xFFFFFFFFu, acc);
    }
}

// The expanded node's neighbour ids, this lane's share of its vector and,
// with the neighbour-code layout (NC), the code rows of this lane's
// neighbours (slots lane + 32 r, two 16-byte chunks each).
template <int DT, int RPL, int DCH, bool NC = false> struct NodeData {
    uint32_t nb[RPL];
    VecShare<DT, DCH> x;
    uint4 code[NC ? 2 * RPL : 1];
};

template <int DT, int RPL, int DCH, bool WITH_VECTOR, bool NC>
__device__ __forceinline__ void load_node(const SearchArgs &a, uint32_t u, int lane,
                                          NodeData<DT, RPL, DCH, NC> &nd)
{
    using E = typename Elem<DT>::T;
    const uint32_t W = a.adj_bits ? a.adj_row_words : a.R;     // words per row
    const uint32_t *row = a.adj + static_cast<uint64_t>(u) * a.adj_stride;
#pragma unroll
    for (int r = 0; r < RPL; ++r) {
        uint32_t i = static_cast<uint32_t>(lane + kWarp * r);
        nd.nb[r] = i < W ? row[i] : kNone;
    }
    if (WITH_VECTOR && !a.cand) {     // staged re-rank: the vectors are read after the search
        const E *x = static_cast<const E *>(a.base) + static_cast<uint64_t>(u) * a.vstride;
        load_share<DT, DCH>(x, a.d, a.vecb_ok != 0, lane, nd.x);
    }
    if constexpr (NC) {
        const uint4 *c = reinterpret_cast<const uint4 *>(a.ncodes) + static_cast<uint64_t>(u) * a.R * 2u;
#pragma unroll
        for (int r = 0; r < RPL; ++r) {
            const uint32_t i = static_cast<uint32_t>(lane + kWarp * r);
            nd.code[2 * r] = i < a.R ? __ldg(c + 2u * i) : make_uint4(0u, 0u, 0u, 0u);
            nd.code[2 * r + 1] = i < a.R ? __ldg(c + 2u * i + 1u) : make_uint4(0u, 0u, 0u, 0u);
        }
    }
}

// Packed rows: neighbour r occupies bits [r*b, r*b + b) of the row's word
// stream (little-endian), all ones meaning an empty slot.  Lane l holds words
// l + 32 t in nb[t]; each lane gathers the two words its ids straddle with
// shuffles and leaves ids (or kNone) in nb.
template <int RPL>
__device__ __forceinline__ void unpack_ids(const SearchArgs &a, int lane, uint32_t (&nb)[RPL])
{
    if (!a.adj_bits) return;
    const uint32_t b = a.adj_bits, mask = (1u << b) - 1u;
    uint32_t w[RPL];
#pragma unroll
    for (int t = 0; t < RPL; ++t) w[t] = nb[t];
#pragma unroll
    for (int t = 0; t < RPL; ++t) {
        const uint32_t r = static_cast<uint32_t>(lane + kWarp * t);
        const uint32_t bit = r * b, wi = bit >> 5, o = bit & 31u;
        uint32_t lo = 0, hi = 0;
        // ids r < 32(t + 1) of at most 32 bits lie in words below 32(t + 1)
#pragma unroll
        for (int s = 0; s <= t; ++s) {
            const uint32_t v0 = __shfl_sync(0xFFFFFFFFu, w[s], static_cast<int>(wi & 31u));
            const uint32_t v1 = __shfl_sync(0xFFFFFFFFu, w[s], static_cast<int>((wi + 1u) & 31u));
            if (static_cast<uint32_t>(s) == (wi >> 5)) lo = v0;
            if (static_cast<uint32_t>(s) == ((wi + 1u) >> 5)) hi = v1;
        }
        const uint32_t v = ((lo >> o) | (o ? hi << (32u - o) : 0u)) & mask;
        nb[t] = (r < a.R && v != mask) ? v : kNone;
    }
}

template <int MODE> __device__ __forceinline__ void store_entry(void *Ts, uint32_t c, float v)
{
    if (MODE == kModeBF16) static_cast<uint16_t *>(Ts)[c] = __bfloat16_as_ushort(__float2bfloat16_rn(v));
    else static_cast<float *>(Ts)[c] = v;
}

// FP32 table entries T[s][c] of one subspace for the centroids
// c = lane + 32 t, t < 8 (§4.1), in the fixed order described above.
__device__ __forceinline__ void subspace_entries(const SearchArgs &a, const float *qv,
                                                 const uint32_t *offs, uint32_t s, int lane,
                                                 float (&v)[8])
{
    const uint32_t o = offs[s], ds = offs[s + 1] - o;
    const float *cb = a.codebook + 256u * o;
    if (ds == 4 && (o & 3u) == 0) {
        const float4 q4 = *reinterpret_cast<const float4 *>(qv + o);
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            const uint32_t c = lane + kWarp * t;
            const float4 c4 = __ldg(reinterpret_cast<const float4 *>(cb) + c);
            float acc = 0.0f, df;
            df = __fsub_rn(q4.x, c4.x); acc = __fmaf_rn(df, df, acc);
            df = __fsub_rn(q4.y, c4.y); acc = __fmaf_rn(df, df, acc);
            df = __fsub_rn(q4.z, c4.z); acc = __fmaf_rn(df, df, acc);
            df = __fsub_rn(q4.w, c4.w); acc = __fmaf_rn(df, df, acc);
            v[t] = acc;
        }
    } else if (ds == 2 && (o & 1u) == 0) {
        const float2 q2 = *reinterpret_cast<const float2 *>(qv + o);
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            const uint32_t c = lane + kWarp * t;
            const float2 c2 = __ldg(reinterpret_cast<const float2 *>(cb) + c);
            float acc = 0.0f, df;
            df = __fsub_rn(q2.x, c2.x); acc = __fmaf_rn(df, df, acc);
            df = __fsub_rn(q2.y, c2.y); acc = __fmaf_rn(df, df, acc);
            v[t] = acc;
        }
    } else {
#pragma unroll 2
        for (int t = 0; t < 8; ++t) {
            const uint32_t c = lane + kWarp * t;
            const float *cc = cb + c * ds;
            float acc = 0.0f;
            for (uint32_t j = 0; j < ds; ++j) {
                float df = __fsub_rn(qv[o + j], __ldg(cc + j));
                acc = __fmaf_rn(df, df, acc);
            }
            v[t] = acc;
        }
    }
}

// PQ distance table of one query into shared memory (§4.1); entries are
// computed in FP32 and stored in the mode's precision.  The 8-bit table takes
// two passes: the first finds each subspace's smallest entry lo_s and the
// widest subspace's range g, the second stores
// min(255, rint((T[s][c] - lo_s) * (255 / g))), each operation rounded to
// FP32 (every entry 0 when g is 0).  Entries are >= +0, so their bit
// patterns order like their values.
template <int MODE>
__device__ __forceinline__ void build_table(const SearchArgs &a, const float *qv,
                                            const uint32_t *offs, void *T, float *lo, int lane,
                                            uint32_t nsub)
{
    float v[8];
    if constexpr (MODE == kModeQ8) {
        float g = 0.0f;
        for (uint32_t s = 0; s < a.M; ++s) {
            subspace_entries(a, qv, offs, s, lane, v);
            uint32_t mn = __float_as_uint(v[0]), mx = mn;
#pragma unroll
            for (int t = 1; t < 8; ++t) {
                const uint32_t b = __float_as_uint(v[t]);
                mn = b < mn ? b : mn;
                mx = b > mx ? b : mx;
            }
            const float fmn = __uint_as_float(__reduce_min_sync(0xFFFFFFFFu, mn));
            const float fmx = __uint_as_float(__reduce_max_sync(0xFFFFFFFFu, mx));
            if (lane == 0) lo[s] = fmn;
            const float w = __fsub_rn(fmx, fmn);
            g = w > g ? w : g;
        }
        __syncwarp();
        const float inv = g > 0.0f ? __fdiv_rn(255.0f, g) : 0.0f;
        for (uint32_t s = 0; s < a.M; ++s) {
            subspace_entries(a, qv, offs, s, lane, v);
            const float los = lo[s];
            uint8_t *Ts = static_cast<uint8_t *>(T) + s * 256u;
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                uint32_t qv8 = 0;
                if (g > 0.0f) {
                    qv8 = __float2uint_rn(__fmul_rn(__fsub_rn(v[t], los), inv));
                    qv8 = qv8 < 255u ? qv8 : 255u;
                }
                Ts[lane + kWarp * t] = static_cast<uint8_t>(qv8);
            }
        }
    } else {
        for (uint32_t s = 0; s < nsub; ++s) {       // nsub < M: the first nsub subspaces only
            subspace_entries(a, qv, offs, s, lane, v);
            unsigned char *Ts = static_cast<unsigned char *>(T) + s * 256u * (MODE == kModeBF16 ? 2u : 4u);
#pragma unroll
            for (int t = 0; t < 8; ++t) store_entry<MODE>(Ts, lane + kWarp * t, v[t]);
        }
    }
}

template <bool ON> struct PhaseClock {
    unsigned long long t, acc[ON ? kPhases : 1];
    __device__ __forceinline__ PhaseClock() : t(0)
    {
#pragma unroll
        for (int i = 0; i < (ON ? kPhases : 1); ++i) acc[i] = 0;
        if constexpr (ON) t = clock64();
    }
    __device__ __forceinline__ void mark(int ph)
    {
        if constexpr (ON) {
            const unsigned long long now = clock64();
            acc[ph] += now - t;
            t = now;
        }
    }
};

// CS, where the new neighbours' code rows come from: 0 = each requested
// after the seen filter (only the new ones); 1 = the neighbour-code layout
// (every neighbour's row arrives with the node); 2 = every neighbour's row
// requested from the codes as soon as the node's row arrives, so that the
// filter runs while they are in flight (rows of at most 32 bytes).
template <int DT, int RPL, int DCH, int MODE, int CS, bool PH>
__global__ void __launch_bounds__(32) search_kernel(const SearchArgs a)
{
    using E = typename Elem<DT>::T;
    constexpr bool kPQ = MODE != kModeExact;
    constexpr bool NC = CS == 1;
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x;
    const SmemLayout lay(a.M, a.log2z, a.L, a.k, a.d, a.R, MODE, a.ntab);
    void *T = smem + lay.off_T;
    uint32_t *bloom = reinterpret_cast<uint32_t *>(smem + lay.off_bloom);
    uint64_t *Lk = reinterpret_cast<uint64_t *>(smem + lay.off_L);
    uint64_t *Nk = reinterpret_cast<uint64_t *>(smem + lay.off_Nk);
    uint32_t *Nid = reinterpret_cast<uint32_t *>(smem + lay.off_Nid);
    uint64_t *Ck = reinterpret_cast<uint64_t *>(smem + lay.off_Ck);
    float *qv = reinterpret_cast<float *>(smem + lay.off_q);
    uint32_t *offs = reinterpret_cast<uint32_t *>(smem + lay.off_offs);
    float *lo8 = reinterpret_cast<float *>(smem + lay.off_lo);

    const uint32_t d = a.d, kstride = a.k;
    const uint32_t zmask = (1u << a.log2z) - 1u;
    const uint32_t nwords = (1u << a.log2z) >= 32u ? (1u << a.log2z) / 32u : 1u;

    uint32_t next_static = blockIdx.x;
    for (;;) {
        // ---- next query: from the work counter (persistent launch) or by grid stride
        uint32_t qi;
        if (a.queue) {
            uint32_t t = 0;
            if (lane == 0) t = atomicAdd(a.queue, 1u);
            qi = __shfl_sync(0xFFFFFFFFu, t, 0);
        } else {
            qi = next_static;
            next_static += gridDim.x;
        }
        if (qi >= a.nq) break;
        const uint32_t q = a.order ? a.order[qi] : qi;
        const uint32_t k = a.k_per_q ? a.k_per_q[q] : a.k;
        const uint32_t L = a.L_per_q ? a.L_per_q[q] : a.L;
        const bool regk = k <= static_cast<uint32_t>(kRegK);
        if (k == 0 || k > a.k || L < k || L > a.L) {     // per-query arguments out of range
            for (uint32_t i = lane; i < kstride; i += kWarp) {
                a.out_ids[static_cast<uint64_t>(q) * kstride + i] = kNone;
                a.out_dist[static_cast<uint64_t>(q) * kstride + i] = __uint_as_float(0x7F800000u);
            }
            if (lane == 0) {
                if (a.out_iters) a.out_iters[q] = 0;
                if (a.out_status) a.out_status[q] = -1;
                if (a.out_ndist) a.out_ndist[q] = 0;
                if (a.cand_n) a.cand_n[q] = 0;
            }
            __syncwarp();
            continue;
        }
        const uint32_t iter_cap = a.iter_cap ? a.iter_cap : 8u * L + 64u;
        PhaseClock<PH> clk;
        const unsigned long long t_start = clk.t;
        // ---- query: FP32 copy in shared memory, this lane's share in registers
        const E *qp = static_cast<const E *>(a.queries) + static_cast<uint64_t>(q) * d;
        if (kPQ) {
            for (uint32_t j = lane; j < d; j += kWarp) qv[j] = static_cast<float>(qp[j]);
            for (uint32_t i = lane; i <= a.M; i += kWarp) offs[i] = a.off[i];
        }
        VecShare<DT, DCH> qs;
        load_share<DT, DCH>(qp, d, a.vec_ok != 0, lane, qs);
        for (uint32_t w = lane; w < nwords; w += kWarp) bloom[w] = 0u;
        __syncwarp();
        bool table_failed = false;
        if ((MODE == kModeBF16 || MODE == kModeF32) && a.tables) {   // precomputed on the tensor cores
            constexpr uint32_t esz = MODE == kModeBF16 ? 2u : 4u;      // BF16 or FP32 entries
            table_failed = *a.tables_err != 0u;
            const uint4 *src = reinterpret_cast<const uint4 *>(static_cast<const unsigned char *>(a.tables) +
                                                               static_cast<uint64_t>(q) * a.M * 256u * esz);
            uint4 *dst = reinterpret_cast<uint4 *>(T);
            for (uint32_t i = lane; i < a.M * 256u * esz / 16u; i += kWarp) dst[i] = src[i];
        } else if (MODE == kModeF32Lazy) {             // the kept subspaces' entries, in FP32
            build_table<kModeF32>(a, qv, offs, T, lo8, lane, a.ntab < a.M ? a.ntab : a.M);
        } else if (kPQ) {
            build_table<MODE>(a, qv, offs, T, lo8, lane, a.M);
        }
        __syncwarp();
        const TableRef tr{T, qv, offs, a.codebook, a.d % a.M == 0 ? a.d / a.M : 0u,
                          MODE == kModeF32Lazy ? a.ntab : a.M};
        clk.mark(kPhTable);

        // ---- start: worklist = {medoid}, medoid marked seen
        const uint32_t s0 = a.entry ? a.entry[q] : a.medoid;
        uint32_t dm_bits = 0;
        if (!kPQ) {
            VecShare<DT, DCH> xs;
            load_share<DT, DCH>(static_cast<const E *>(a.base) + static_cast<uint64_t>(s0) * a.vstride, d,
                                a.vecb_ok != 0, lane, xs);
            dm_bits = exact_distance_bits<DT, DCH>(qs, xs);
        }
        if (lane == 0) {
            const uint32_t s = s0;
            if (kPQ)
                dm_bits = pq_dist_bits<MODE>(tr, a.codes + static_cast<uint64_t>(s) * a.Mpad, a.M, a.Mpad);
            Lk[0] = make_key(dm_bits, s);
            uint32_t p1 = fnv1a32_id(s) & zmask, p2 = fnv1a64_id_folded(s) & zmask;
            bloom[p1 >> 5] |= 1u << (p1 & 31u);
            bloom[p2 >> 5] |= 1u << (p2 & 31u);
        }
        uint32_t nl = 1, nc = 0, iters = 0, ndist = 1, first = 0;
        bool have_next = !table_failed;
        int32_t status = table_failed ? 2 : 0;
        uint64_t ck = ~0ull;               // register top-k (k <= kRegK): lane i holds rank i
        uint32_t cur = s0;
        NodeData<DT, RPL, DCH, NC> nd, nd2;   // nd2: the speculative request (a.spec)
        load_node<DT, RPL, DCH, kPQ, NC>(a, cur, lane, nd);
        __syncwarp();

        while (have_next) {
            if (iters >= iter_cap) {
                status = 1;
                break;
            }
            // u* = first unvisited entry of the sorted worklist (Alg. 1); its
            // position comes out of the previous merge
            const uint64_t ukey = Lk[first];
            const uint32_t u = key_id(ukey);
            __syncwarp();
            if (lane == 0) {
                Lk[first] = ukey | 1ull;
                if (a.trace && iters < a.trace_cap)
                    a.trace[static_cast<uint64_t>(q) * a.trace_cap + iters] = u;
                if (a.cand && !a.cand_list && iters < a.cand_cap)
                    a.cand[static_cast<uint64_t>(q) * a.cand_cap + iters] = u;
            }
            ++iters;
            if (u != cur) {  // the prefetched node is always u*; reload if not
                cur = u;
                load_node<DT, RPL, DCH, kPQ, NC>(a, cur, lane, nd);
            }
            // the first unvisited worklist entry after u*: one of the two
            // candidates for the next node (§4.5); with a.spec its lists are
            // requested now, before this iteration's distances are known
            uint64_t lkey = ~0ull;
            int lnext = -1;                  // index of that worklist entry
            for (uint32_t b0 = first + 1; b0 < nl; b0 += kWarp) {
                const uint32_t i = b0 + lane;
                const bool v = i < nl && !(Lk[i] & 1ull);
                const uint32_t bal = __ballot_sync(0xFFFFFFFFu, v);
                if (bal) {
                    lnext = static_cast<int>(b0 + __ffs(bal) - 1);
                    lkey = Lk[lnext];
                    break;
                }
            }
            if (a.spec && lkey != ~0ull) load_node<DT, RPL, DCH, kPQ, NC>(a, key_id(lkey), lane, nd2);
            VecShare<DT, DCH> xu;                // u*'s vector, for the re-rank below (PQ modes)
            clk.mark(kPhSelect);

            unpack_ids<RPL>(a, lane, nd.nb);
            // early code rows (CS 2): every neighbour's row requested now
            uint4 ec[CS == 2 ? 2 * RPL : 1];
            if constexpr (CS == 2) {
#pragma unroll
                for (int r = 0; r < RPL; ++r) {
                    const uint32_t id = nd.nb[r];
                    const uint4 *row16 = reinterpret_cast<const uint4 *>(
                        a.codes + static_cast<uint64_t>(id == kNone ? 0u : id) * a.Mpad);
                    ec[2 * r] = id != kNone ? __ldg(row16) : make_uint4(0u, 0u, 0u, 0u);
                    ec[2 * r + 1] = (id != kNone && a.Mpad > 16u) ? __ldg(row16 + 1) : make_uint4(0u, 0u, 0u, 0u);
                }
            }
            // ---- filter seen neighbours, §4.3: test all, then insert all
            bool fresh[RPL];
            uint32_t p1[RPL], p2[RPL], slot[RPL];
#pragma unroll
            for (int r = 0; r < RPL; ++r) {
                const uint32_t id = nd.nb[r];
                fresh[r] = false;
                p1[r] = p2[r] = 0;
                if (id != kNone) {
                    p1[r] = fnv1a32_id(id) & zmask;
                    p2[r] = fnv1a64_id_folded(id) & zmask;
                    const uint32_t w1 = bloom[p1[r] >> 5], w2 = bloom[p2[r] >> 5];   // both loads at once
                    const bool hit = (w1 >> (p1[r] & 31u)) & (w2 >> (p2[r] & 31u)) & 1u;
                    fresh[r] = !hit;
                }
            }
            __syncwarp();
            uint32_t nn = 0;
#pragma unroll
            for (int r = 0; r < RPL; ++r) {
                if (fresh[r]) {
                    atomicOr(&bloom[p1[r] >> 5], 1u << (p1[r] & 31u));
                    atomicOr(&bloom[p2[r] >> 5], 1u << (p2[r] & 31u));
                }
                const uint32_t bal = __ballot_sync(0xFFFFFFFFu, fresh[r]);
                slot[r] = nn + __popc(bal & ((1u << lane) - 1u));
                if (fresh[r]) Nid[slot[r]] = nd.nb[r];
                nn += __popc(bal);
            }
            __syncwarp();
            clk.mark(kPhFilter);

            // ---- distances of the new neighbours: PQ (§4.4), one lane per
            // neighbour; or exact (§5.2), the warp per neighbour, four
            // neighbours' vectors requested at a time
            // Keys of the new neighbours: in registers where one lane computed
            // them (kk[t], valid where kv[t]), otherwise in Nk[0..nn).
            uint64_t kk[RPL];
            bool kv[RPL];
#pragma unroll
            for (int t = 0; t < RPL; ++t) {
                kk[t] = ~0ull;
                kv[t] = false;
            }
            bool in_regs = false;
            if constexpr (NC) {              // code rows arrived with the node: the lane that holds them
#pragma unroll
                for (int r = 0; r < RPL; ++r) {
                    if (!fresh[r]) continue;
                    const uint4 c0 = nd.code[2 * r], c1 = nd.code[2 * r + 1];
                    Nk[slot[r]] = make_key(pq_dist_bits_g<MODE>(tr, [c0, c1](uint32_t c16) { return c16 ? c1 : c0; },
                                                                a.M, a.Mpad), nd.nb[r]);
                }
            } else if constexpr (CS == 2) {   // code rows requested before the filter
                // compacted: new neighbour j goes to lane j % 32, which takes
                // its code row from the lane that loaded it (shuffles), so a
                // pass computes up to 32 distances instead of one per slot
                in_regs = true;
                uint32_t *src = reinterpret_cast<uint32_t *>(Nk);    // scratch until the keys
#pragma unroll
                for (int r = 0; r < RPL; ++r)
                    if (fresh[r]) src[slot[r]] = static_cast<uint32_t>(lane) | (static_cast<uint32_t>(r) << 5);
                __syncwarp();
#pragma unroll
                for (int t = 0; t < RPL; ++t) {
                    if (static_cast<uint32_t>(kWarp * t) >= nn) break;           // warp-uniform
                    const uint32_t j = lane + kWarp * t;
                    const uint32_t sv = j < nn ? src[j] : 0u;
                    const int sl = static_cast<int>(sv & 31u);
                    const uint32_t sr = sv >> 5;
                    uint4 c0 = make_uint4(0u, 0u, 0u, 0u), c1 = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
                    for (int r = 0; r < RPL; ++r) {
                        uint4 v0, v1;
                        v0.x = __shfl_sync(0xFFFFFFFFu, ec[2 * r].x, sl);
                        v0.y = __shfl_sync(0xFFFFFFFFu, ec[2 * r].y, sl);
                        v0.z = __shfl_sync(0xFFFFFFFFu, ec[2 * r].z, sl);
                        v0.w = __shfl_sync(0xFFFFFFFFu, ec[2 * r].w, sl);
                        if (a.Mpad > 16u) {                                      // uniform
                            v1.x = __shfl_sync(0xFFFFFFFFu, ec[2 * r + 1].x, sl);
                            v1.y = __shfl_sync(0xFFFFFFFFu, ec[2 * r + 1].y, sl);
                            v1.z = __shfl_sync(0xFFFFFFFFu, ec[2 * r + 1].z, sl);
                            v1.w = __shfl_sync(0xFFFFFFFFu, ec[2 * r + 1].w, sl);
                        } else {
                            v1 = make_uint4(0u, 0u, 0u, 0u);
                        }
                        if (sr == static_cast<uint32_t>(r)) {
                            c0 = v0;
                            c1 = v1;
                        }
                    }
                    if (j < nn) {
                        const uint32_t id = Nid[j];
                        kk[t] = make_key(pq_dist_bits_g<MODE>(tr, [c0, c1](uint32_t c16) { return c16 ? c1 : c0; },
                                                              a.M, a.Mpad), id);
                        kv[t] = true;
                    }
                }
            } else if (kPQ) {
                in_regs = true;
                if (MODE == kModeQ8 && nn <= 8u) {           // exact integer sums: split each row
                    pq_q8_split<4>(a, static_cast<const uint8_t *>(T), Nid, nn, lane, kk[0], kv[0]);
                } else if (MODE == kModeQ8 && nn <= 16u) {
                    pq_q8_split<2>(a, static_cast<const uint8_t *>(T), Nid, nn, lane, kk[0], kv[0]);
                } else {
#pragma unroll
                    for (int t = 0; t < RPL; ++t) {
                        const uint32_t j = lane + kWarp * t;
                        if (j < nn) {
                            const uint32_t id = Nid[j];
                            kk[t] = make_key(pq_dist_bits<MODE>(tr, a.codes + static_cast<uint64_t>(id) * a.Mpad,
                                                                a.M, a.Mpad), id);
                            kv[t] = true;
                        }
                    }
                }
            } else if (DT != 2 && DCH == 1 && (d & 15u) == 0 && a.vecb_ok) {
                // integer data sums exactly in any order, so one lane takes
                // one new neighbour (its whole row) and all of them are
                // requested at once; query words come by shuffle
                const uint32_t nw = d / 4u;  // 32-bit words per row, <= 32
                for (uint32_t j0 = 0; j0 < nn; j0 += kWarp) {
                    const uint32_t j = j0 + static_cast<uint32_t>(lane);
                    const bool act = j < nn;
                    const uint32_t id = act ? Nid[j] : 0u;
                    const uint4 *row = reinterpret_cast<const uint4 *>(static_cast<const E *>(a.base) +
                                                                       static_cast<uint64_t>(id) * a.vstride);
                    uint4 xv[8];
#pragma unroll
                    for (int c = 0; c < 8; ++c)
                        xv[c] = (act && 4u * c < nw) ? __ldg(row + c) : make_uint4(0u, 0u, 0u, 0u);
                    uint32_t acc = 0;
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        const uint32_t xw[4] = {xv[c].x, xv[c].y, xv[c].z, xv[c].w};
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            const uint32_t w = 4u * c + i;
                            const uint32_t qw = __shfl_sync(0xFFFFFFFFu, qs.w[0], static_cast<int>(w));
                            const uint32_t x = DT == 1 ? xw[i] ^ 0x80808080u : xw[i];
                            if (w < nw) {
                                const uint32_t df = __vabsdiffu4(qw, x);
                                acc = __dp4a(df, df, acc);
                            }
                        }
                    }
                    if (act) Nk[j] = make_key(acc, id);
                }
            } else {
                for (uint32_t j0 = 0; j0 < nn; j0 += 4) {
                    VecShare<DT, DCH> xs[4];
                    uint32_t ids[4];
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        ids[t] = j0 + t < nn ? Nid[j0 + t] : 0u;
                        if (j0 + t < nn)
                            load_share<DT, DCH>(static_cast<const E *>(a.base) + static_cast<uint64_t>(ids[t]) * a.vstride,
                                                d, a.vecb_ok != 0, lane, xs[t]);
                    }
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        if (j0 + t < nn) {
                            const uint32_t e = exact_distance_bits<DT, DCH>(qs, xs[t]);
                            if (lane == 0) Nk[j0 + t] = make_key(e, ids[t]);
                        }
                    }
                }
            }
            ndist += nn;
            __syncwarp();
            if (!in_regs) {
#pragma unroll
                for (int t = 0; t < RPL; ++t) {
                    const uint32_t j = lane + kWarp * t;
                    kv[t] = j < nn;
                    kk[t] = kv[t] ? Nk[j] : ~0ull;
                }
                __syncwarp();
            }
            // New keys behind the last entry of a full worklist land at L or
            // later, and so does every larger key: drop them here, so that
            // only keys that enter the list are merged (§4.6-§4.7); the rest
            // are compacted into Nk[0..nm).
            uint32_t nm = 0;
            uint64_t bestn = ~0ull;
            {
                const uint64_t last = nl == L ? Lk[L - 1] >> 1 : ~0ull;
#pragma unroll
                for (int t = 0; t < RPL; ++t) {
                    const bool keep = kv[t] && (kk[t] >> 1) < last;
                    const uint32_t bal = __ballot_sync(0xFFFFFFFFu, keep);
                    if (keep) {
                        Nk[nm + __popc(bal & ((1u << lane) - 1u))] = kk[t];
                        bestn = kk[t] < bestn ? kk[t] : bestn;
                    }
                    nm += __popc(bal);
                }
            }
            __syncwarp();
            clk.mark(kPhDistance);

            // ---- eager next node, §4.5: the best of the new neighbours and
            // the first unvisited worklist entry after u*; prefetch its lists.
            // A dropped key is never the best: the first unvisited entry, if
            // any, precedes it, and otherwise the search ends in the merge.
            uint64_t best = ~0ull;
            {
                best = lkey < bestn ? lkey : bestn;
                best = warp_min_key(best);
                if (kPQ) xu = nd.x;              // wait for the vector only here
                if (best != ~0ull) {
                    cur = key_id(best);
                    if (a.spec && best == lkey) nd = nd2;           // requested at the start
                    else load_node<DT, RPL, DCH, kPQ, NC>(a, cur, lane, nd);
                }
            }
            clk.mark(kPhNext);
            // ---- re-rank candidate: exact distance of u* (§4.8), off the
            // critical path: the next node's lists are already requested
            // (staged re-rank: recorded above, ranked by rerank_kernel)
            if (kPQ && !a.cand) {
                const uint64_t e = make_key(exact_distance_bits<DT, DCH>(qs, xu), u);
                if (regk) {
                    const uint32_t pos = __popc(__ballot_sync(0xFFFFFFFFu, ck < e));
                    if (pos < k) {
                        const uint64_t up = shfl_up_u64(ck, 1);
                        if (static_cast<uint32_t>(lane) == pos) ck = e;
                        else if (static_cast<uint32_t>(lane) > pos) ck = up;
                    }
                    nc = nc + 1 < k ? nc + 1 : k;
                } else if (!(nc == k && e >= Ck[k - 1])) {
                    uint32_t less = 0;
                    uint64_t keep[kMaxK / kWarp];
#pragma unroll
                    for (int t = 0; t < kMaxK / kWarp; ++t) {
                        uint32_t i = lane + kWarp * t;
                        keep[t] = i < nc ? Ck[i] : 0ull;
                        less += (i < nc && keep[t] < e) ? 1u : 0u;
                    }
                    const uint32_t pos = __reduce_add_sync(0xFFFFFFFFu, less);
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
            clk.mark(kPhRerank);

            // ---- merge the new neighbours into the worklist, §4.6-§4.7.
            // Output position = own index + rank in the other list (keys are
            // unique: a new neighbour was never seen, so its id is not in the
            // list).  A new key's rank in the worklist comes from a 4-ary
            // search, its rank among the new keys from a count; its output
            // position is marked in a bit mask.  Every other output position
            // p takes worklist entry p - (new keys before p): entries move
            // right only, so groups of up to 8 chunks are read, then written,
            // from the end of the list down to the first insertion point.
            uint32_t npos = 0;               // new position of `best`, plus one
            if (nm > 0) {
                uint32_t *obits = Nid;       // ids are in the keys now: output-position bits (L <= 1024)
                const uint32_t nl2 = nl + nm < L ? nl + nm : L;
                const uint32_t nw = (nl2 + 31u) >> 5;
                if (static_cast<uint32_t>(lane) < nw) obits[lane] = 0u;
                uint64_t xk[RPL];
                uint32_t xpos[RPL];
                uint32_t rmin = 0xFFFFFFFFu;
                const uint32_t b4 = 1u << ((31 - __clz(nl)) & ~1);     // largest power of 4 <= nl
#pragma unroll
                for (int t = 0; t < RPL; ++t) {
                    const uint32_t j = lane + kWarp * t;
                    xk[t] = 0;
                    xpos[t] = 0xFFFFFFFFu;
                    if (j < nm) {
                        const uint64_t x = Nk[j];
                        uint32_t lo = 0;     // #{worklist keys < x}
                        for (uint32_t b = b4; b != 0u; b >>= 2) {
                            const uint32_t c1 = lo + b, c2 = c1 + b, c3 = c2 + b;
                            const uint32_t m = static_cast<uint32_t>(c1 <= nl && Lk[c1 - 1u] < x) +
                                               static_cast<uint32_t>(c2 <= nl && Lk[c2 - 1u] < x) +
                                               static_cast<uint32_t>(c3 <= nl && Lk[c3 - 1u] < x);
                            lo += b * m;
                        }
                        uint32_t rn = 0, tt = 0;
                        for (; tt + 4 <= nm; tt += 4)
                            rn += (Nk[tt] < x) + (Nk[tt + 1] < x) + (Nk[tt + 2] < x) + (Nk[tt + 3] < x);
                        for (; tt < nm; ++tt) rn += Nk[tt] < x;
                        xk[t] = x;
                        xpos[t] = lo + rn;
                        rmin = lo < rmin ? lo : rmin;
                    }
                }
                rmin = __reduce_min_sync(0xFFFFFFFFu, rmin);
                __syncwarp();
#pragma unroll
                for (int t = 0; t < RPL; ++t)
                    if (xpos[t] < L) atomicOr(&obits[xpos[t] >> 5], 1u << (xpos[t] & 31u));
                __syncwarp();
                // lane c: the new keys' positions in chunk c, and how many lie below it
                const uint32_t wbits = static_cast<uint32_t>(lane) < nw ? obits[lane] : 0u;
                uint32_t pre = __popc(wbits);
#pragma unroll
                for (int h = 1; h < kWarp; h <<= 1) {
                    const uint32_t v = __shfl_up_sync(0xFFFFFFFFu, pre, h);
                    if (lane >= h) pre += v;
                }
                pre -= __popc(wbits);
                clk.mark(kPhMergeRank);
                const int32_t cmin = static_cast<int32_t>(rmin >> 5);
                const uint32_t lt = (1u << lane) - 1u;
                for (int32_t ctop = static_cast<int32_t>(nw) - 1; ctop >= cmin; ctop -= 8) {
                    uint64_t key[8];
                    uint32_t dst[8];
#pragma unroll
                    for (int g = 0; g < 8; ++g) {
                        const int32_t c = ctop - g;
                        key[g] = 0;
                        dst[g] = 0xFFFFFFFFu;
                        if (c >= cmin) {
                            const uint32_t w = __shfl_sync(0xFFFFFFFFu, wbits, c);
                            const uint32_t below = __shfl_sync(0xFFFFFFFFu, pre, c) + __popc(w & lt);
                            const uint32_t p = static_cast<uint32_t>(c) * 32u + lane;
                            if (p < nl2 && p >= rmin && !((w >> lane) & 1u)) {
                                key[g] = Lk[p - below];
                                dst[g] = p;
                                if (key[g] == best) npos = p + 1;
                            }
                        }
                    }
                    __syncwarp();
#pragma unroll
                    for (int g = 0; g < 8; ++g)
                        if (dst[g] != 0xFFFFFFFFu) Lk[dst[g]] = key[g];
                    __syncwarp();
                }
                clk.mark(kPhMergeShift);
#pragma unroll
                for (int t = 0; t < RPL; ++t) {
                    if (xpos[t] < L) {
                        Lk[xpos[t]] = xk[t];
                        if (xk[t] == best) npos = xpos[t] + 1;
                    }
                }
                __syncwarp();
                nl = nl2;
                npos = __reduce_max_sync(0xFFFFFFFFu, npos);
                if (npos == 0 && lnext >= 0 && best == lkey)      // in the untouched prefix
                    npos = static_cast<uint32_t>(lnext) + 1;
            } else if (lnext >= 0) {
                npos = static_cast<uint32_t>(lnext) + 1;
            }
            have_next = npos != 0;
            first = npos - 1;
            clk.mark(kPhMerge);
        }

        // ---- output: re-ranked top-k (§4.8), or in the exact mode the first
        // k worklist entries (Alg. 1's result); padded.  With the staged
        // re-rank only the number of candidates.
        if (kPQ && a.cand) {
            if (a.cand_list) {            // the final worklist (the top-L by PQ distance)
                for (uint32_t i = lane; i < nl; i += kWarp)
                    a.cand[static_cast<uint64_t>(q) * a.cand_cap + i] = key_id(Lk[i]);
                if (lane == 0) a.cand_n[q] = nl;
            } else if (lane == 0) {
                a.cand_n[q] = iters < a.cand_cap ? iters : a.cand_cap;
            }
        } else if (!kPQ) {
            for (uint32_t i = lane; i < kstride; i += kWarp) {
                const uint64_t o = static_cast<uint64_t>(q) * kstride + i;
                if (i < nl && i < k) {
                    const uint64_t key = Lk[i];
                    const uint32_t bits = static_cast<uint32_t>(key >> 32);
                    a.out_ids[o] = key_id(key);
                    a.out_dist[o] = DT == 2 ? __uint_as_float(bits) : static_cast<float>(bits);
                } else {
                    a.out_ids[o] = kNone;
                    a.out_dist[o] = __uint_as_float(0x7F800000u);
                }
            }
        } else if (regk) {
            for (uint32_t i = lane; i < kstride; i += kWarp) {
                const uint64_t o = static_cast<uint64_t>(q) * kstride + i;
                if (i < nc) {                  // nc <= k <= 32: rank i is lane i's register
                    const uint32_t bits = static_cast<uint32_t>(ck >> 32);
                    a.out_ids[o] = key_id(ck);
                    a.out_dist[o] = DT == 2 ? __uint_as_float(bits) : static_cast<float>(bits);
                } else {
                    a.out_ids[o] = kNone;
                    a.out_dist[o] = __uint_as_float(0x7F800000u);
                }
            }
        } else {
            for (uint32_t i = lane; i < kstride; i += kWarp) {
                const uint64_t o = static_cast<uint64_t>(q) * kstride + i;
                if (i < nc) {
                    const uint64_t key = Ck[i];
                    const uint32_t bits = static_cast<uint32_t>(key >> 32);
                    a.out_ids[o] = key_id(key);
                    a.out_dist[o] = DT == 2 ? __uint_as_float(bits) : static_cast<float>(bits);
                } else {
                    a.out_ids[o] = kNone;
                    a.out_dist[o] = __uint_as_float(0x7F800000u);
                }
            }
        }
        if constexpr (PH) {
            if (lane == 0) {
                clk.acc[kPhTotal] = clock64() - t_start;
#pragma unroll
                for (int i = 0; i < kPhases; ++i)
                    a.phase_cycles[static_cast<uint64_t>(q) * kPhases + i] = clk.acc[i];
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

// Launch for one mode: dispatch on element type, neighbours per lane
// (R <= 64 or <= 128) and 128-dimension chunks per lane (d <= 128 or <= 512).
template <int DT, int RPL, int DCH, int MODE, int CS, bool PH>
cudaError_t launch_one(const SearchArgs &a, size_t smem, cudaStream_t st)
{
    cudaError_t e = cudaFuncSetAttribute(search_kernel<DT, RPL, DCH, MODE, CS, PH>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    if (e != cudaSuccess) return e;
    // the carve-out is a hint that stays with the function: set it when the
    // request changes (back to the CUDA driver's choice, -1, when it is 0)
    static std::atomic<uint32_t> carveout_set{0};
    if (carveout_set.load() != a.carveout) {
        e = cudaFuncSetAttribute(search_kernel<DT, RPL, DCH, MODE, CS, PH>,
                                 cudaFuncAttributePreferredSharedMemoryCarveout,
                                 a.carveout ? static_cast<int>(a.carveout) : -1);
        if (e != cudaSuccess) return e;
        carveout_set.store(a.carveout);
    }
    uint32_t grid = a.nq;
    if (a.queue) {                     // persistent: a multiple of the resident CTAs
        int dev = 0, sms = 0, per_sm = 0;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
        if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, search_kernel<DT, RPL, DCH, MODE, CS, PH>,
                                                               32, smem)) != cudaSuccess)
            return e;
        const uint64_t want = static_cast<uint64_t>(sms) * (per_sm > 0 ? per_sm : 1) *
                              (a.grid_mult ? a.grid_mult : 1u);
        grid = static_cast<uint32_t>(want < a.nq ? want : a.nq);
    }
    search_kernel<DT, RPL, DCH, MODE, CS, PH><<<grid, 32, smem, st>>>(a);
    return cudaGetLastError();
}

// The per-phase clock (SearchArgs::phase_cycles) is a separate instantiation,
// so the timed kernel carries none of its registers or branches.
template <int DT, int RPL, int DCH, int MODE, int CS = 0>
cudaError_t launch_ph(const SearchArgs &a, size_t smem, cudaStream_t st)
{
    return a.phase_cycles ? launch_one<DT, RPL, DCH, MODE, CS, true>(a, smem, st)
                          : launch_one<DT, RPL, DCH, MODE, CS, false>(a, smem, st);
}

template <int MODE> cudaError_t launch_mode(const SearchArgs &a, int dtype, size_t smem, cudaStream_t st)
{
    const bool narrow = a.d <= 128, wide_r = a.R > 64;
    if constexpr (MODE != kModeExact) {
        if (a.ncodes) {                // neighbour-code layout: R <= 64, d <= 128, checked by the caller
            if (dtype == 0) return launch_ph<0, 2, 1, MODE, 1>(a, smem, st);
            if (dtype == 1) return launch_ph<1, 2, 1, MODE, 1>(a, smem, st);
            return launch_ph<2, 2, 1, MODE, 1>(a, smem, st);
        }
        if (a.early_codes && !wide_r && narrow && a.Mpad <= 32u) {   // early code rows
            if (dtype == 0) return launch_ph<0, 2, 1, MODE, 2>(a, smem, st);
            if (dtype == 1) return launch_ph<1, 2, 1, MODE, 2>(a, smem, st);
            return launch_ph<2, 2, 1, MODE, 2>(a, smem, st);
        }
    }
#define BANG_DISPATCH(DT)                                                                    \
    return wide_r ? (narrow ? launch_ph<DT, 4, 1, MODE>(a, smem, st) : launch_ph<DT, 4, 4, MODE>(a, smem, st)) \
                  : (narrow ? launch_ph<DT, 2, 1, MODE>(a, smem, st) : launch_ph<DT, 2, 4, MODE>(a, smem, st))
    if (dtype == 0) { BANG_DISPATCH(0); }
    if (dtype == 1) { BANG_DISPATCH(1); }
    BANG_DISPATCH(2);
#undef BANG_DISPATCH
}

// One translation unit per mode instantiates these.
cudaError_t launch_search_f32(const SearchArgs &a, int dtype, size_t smem, cudaStream_t st);
cudaError_t launch_search_bf16(const SearchArgs &a, int dtype, size_t smem, cudaStream_t st);
cudaError_t launch_search_exact(const SearchArgs &a, int dtype, size_t smem, cudaStream_t st);
cudaError_t launch_search_q8(const SearchArgs &a, int dtype, size_t smem, cudaStream_t st);
cudaError_t launch_search_f32lazy(const SearchArgs &a, int dtype, size_t smem, cudaStream_t st);

}  // namespace bang
