// PQ distance tables on the tensor cores (§4.1's PQDistTable as a dense
// queries x centroids contraction), tcgen05 (sm_100 family) form.
//
//   T[q][s][c] = ||q_s||^2 + ||C_s[c]||^2 - 2 q_s . C_s[c]
//
// The cross term is a GEMM per subspace: A = the queries' dimensions of the
// 16-wide K block(s) holding subspace s (128 queries per CTA, BF16), B = the
// 256 centroids of s written into the same 16-wide block with zeros outside
// the subspace's dimensions.  Accuracy: uint8/int8 queries are exact in BF16;
// FP32 queries and the centroids are split into three BF16 parts each (about
// 24 significant bits), and the products that matter (high x all, middle x
// high and middle, low x high) are summed in the FP32 accumulator, which
// gives the cross term to about FP32 accuracy; the norms are FP32.  Tables come out FP32 or
// BF16 (the reduced-precision search form reads BF16 tables).  The TF32 form
// (a.tf32 with centroid tiles rounded to TF32 on the host) rounds both
// operands to TF32 first; a TF32 value is exactly the sum of two BF16 parts,
// so the same MMAs then form exact TF32 x TF32 products with FP32
// accumulation: the numerics of a TF32 GEMM, at about its tensor-pipe cost
// (two BF16 MMAs per TF32 MMA).
//
// Per CTA: 128 threads; thread t owns query row t of the tile (TMEM lane t)
// and writes that row of the query operand for each subspace's K blocks.
// Operands live in shared memory in the no-swizzle K-major layout: 8-row x
// 16-byte core matrices, K-adjacent cores 128 bytes apart, M/N-adjacent
// cores 256 bytes apart.  One thread issues the MMAs; completion is signalled
// through an mbarrier; every wait is bounded and reports failure in *err.
#include <cuda_runtime.h>

#include <cstdint>
#include <cuda_bf16.h>

#include "adc_table_tc.h"

namespace bang {
namespace {

constexpr uint32_t kTile = 128;            // queries per CTA (UMMA M)
constexpr uint32_t kN = 256;               // centroids per subspace (UMMA N)
constexpr uint32_t kACore = 4096;          // bytes of one 128 x 16 BF16 operand
constexpr uint32_t kBCore = 8192;          // bytes of one 256 x 16 BF16 operand
constexpr uint32_t kMaxWaitSpins = 1u << 26;
constexpr uint32_t kSubPerCta = 4;         // subspaces per CTA (grid y covers the rest)

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor: start, leading (K) and stride (M/N) byte
// offsets, fixed version bits for this architecture, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr)
{
    uint64_t d = 0;
    d |= static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4);
    d |= static_cast<uint64_t>(128u >> 4) << 16;   // K-adjacent core matrices
    d |= static_cast<uint64_t>(256u >> 4) << 32;   // M/N-adjacent core matrices
    d |= static_cast<uint64_t>(1u) << 46;
    return d;
}

// Instruction descriptor: FP32 accumulator, BF16 A and B, both K-major,
// N = 256, M = 128.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((kN >> 3) << 17) | ((kTile >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mbar)
                 : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity)
{
    for (uint32_t i = 0; i < kMaxWaitSpins; ++i) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred P;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, P;\n\t}\n"
            : "=r"(ok)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float *v)
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
        "%12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, "
        "%30, %31}, [%32];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
          "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
          "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Round to TF32 (10 mantissa bits), to nearest with ties to even: the
// operands of the TF32 form, whose products the split parts then carry
// exactly (a TF32 value is the sum of two BF16 values).
__device__ __forceinline__ float tf32_rne(float x)
{
    uint32_t u = __float_as_uint(x);
    u += 0xFFFu + ((u >> 13) & 1u);
    return __uint_as_float(u & ~0x1FFFu);
}

// Offset of element (row, k) of a K-major no-swizzle operand with 16 K
// columns: core (row/8, k/8), 8 rows of 16 bytes per core.
__device__ __forceinline__ uint32_t core_off(uint32_t row, uint32_t k)
{
    return ((row >> 3) * 2u + (k >> 3)) * 128u + (row & 7u) * 16u + (k & 7u) * 2u;
}

template <int DT>
__global__ void __launch_bounds__(128) adc_table_tc_kernel(TcTableArgs a)
{
    using E = typename TcElem<DT>::T;
    extern __shared__ __align__(1024) unsigned char smem[];
    const uint32_t t = threadIdx.x, warp = t >> 5;
    // carve: query operand (3 parts x kMaxKbPerSub K blocks x 4 KB), centroid
    // operand (3 parts x kMaxKbPerSub x 8 KB), centroid norms (256 floats),
    // mbarrier, TMEM address
    constexpr uint32_t kAParts = DT == 2 ? 3u : 1u;   // integer queries are exact in BF16
    unsigned char *Abuf = smem;
    unsigned char *Bbuf = Abuf + 3u * kMaxKbPerSub * kACore;
    float *cn = reinterpret_cast<float *>(Bbuf + 3u * kMaxKbPerSub * kBCore);
    uint64_t *mbar = reinterpret_cast<uint64_t *>(cn + kN);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(mbar + 1);

    const uint32_t q0 = blockIdx.x * kTile;
    const uint32_t q = q0 + t;
    const bool valid = q < a.nq;
    const E *qp = static_cast<const E *>(a.queries) + static_cast<uint64_t>(valid ? q : 0u) * a.d;

    if (t == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(mbar)) : "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(kN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    bool ok = true;

    // this CTA's subspaces: group blockIdx.y of kSubPerCta
    const uint32_t s_begin = blockIdx.y * kSubPerCta;
    const uint32_t s_end = s_begin + kSubPerCta < a.M ? s_begin + kSubPerCta : a.M;
    for (uint32_t s = s_begin; s < s_end && ok; ++s) {
        const uint32_t o = a.off[s], ds = a.off[s + 1] - o;
        const uint32_t kb0 = o / 16u, kb1 = (o + ds - 1u) / 16u;
        const uint32_t nb = kb1 - kb0 + 1u;              // <= kMaxKbPerSub (checked on the host)
        if (nb > kMaxKbPerSub) {                         // uniform: every thread sees the same nb
            ok = false;
            break;
        }
        // ---- this thread's query row over the subspace's K blocks (zero
        // beyond d and nq), split into BF16 parts
        for (uint32_t b = 0; b < nb; ++b)
            for (uint32_t kk = 0; kk < 16; ++kk) {
                const uint32_t j = (kb0 + b) * 16u + kk;
                float x = (valid && j < a.d) ? static_cast<float>(qp[j]) : 0.0f;
                if (a.tf32) x = tf32_rne(x);
                const __nv_bfloat16 h = __float2bfloat16_rn(x);
                const float r1 = x - __bfloat162float(h);
                const __nv_bfloat16 m = __float2bfloat16_rn(r1);
                const __nv_bfloat16 l = __float2bfloat16_rn(r1 - __bfloat162float(m));
                const uint32_t e = core_off(t, kk);
                *reinterpret_cast<uint16_t *>(Abuf + (0u * kMaxKbPerSub + b) * kACore + e) = __bfloat16_as_ushort(h);
                if (kAParts > 1) {
                    *reinterpret_cast<uint16_t *>(Abuf + (1u * kMaxKbPerSub + b) * kACore + e) = __bfloat16_as_ushort(m);
                    *reinterpret_cast<uint16_t *>(Abuf + (2u * kMaxKbPerSub + b) * kACore + e) = __bfloat16_as_ushort(l);
                }
            }
        // ---- centroid tiles of subspace s (three parts per K block,
        // prepared at load time) and the norms
        const uint4 *src = reinterpret_cast<const uint4 *>(a.btiles + static_cast<uint64_t>(a.bfirst[s]) * kBCore);
        uint4 *dst = reinterpret_cast<uint4 *>(Bbuf);
        for (uint32_t i = t; i < nb * 3u * kBCore / 16u; i += blockDim.x) dst[i] = src[i];
        for (uint32_t c = t; c < kN; c += blockDim.x) cn[c] = a.cnorm[s * kN + c];
        // make generic-proxy shared stores visible to the tensor cores
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        __syncthreads();
        if (t == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            uint32_t acc = 0;
            for (uint32_t b = 0; b < nb; ++b) {
                const uint64_t ah = smem_desc(smem_u32(Abuf + (0u * kMaxKbPerSub + b) * kACore));
                const uint64_t bh = smem_desc(smem_u32(Bbuf + (3u * b) * kBCore));
                const uint64_t bm = smem_desc(smem_u32(Bbuf + (3u * b + 1u) * kBCore));
                const uint64_t bl = smem_desc(smem_u32(Bbuf + (3u * b + 2u) * kBCore));
                mma_bf16(tmem, ah, bh, acc); acc = 1;
                mma_bf16(tmem, ah, bm, 1);
                mma_bf16(tmem, ah, bl, 1);
                if (kAParts > 1) {
                    const uint64_t am = smem_desc(smem_u32(Abuf + (1u * kMaxKbPerSub + b) * kACore));
                    const uint64_t al = smem_desc(smem_u32(Abuf + (2u * kMaxKbPerSub + b) * kACore));
                    mma_bf16(tmem, am, bh, 1);
                    mma_bf16(tmem, am, bm, 1);
                    mma_bf16(tmem, al, bh, 1);
                }
            }
            mma_commit(smem_u32(mbar));
        }
        // every thread waits with a bound; the vote keeps the outcome uniform
        ok = __syncthreads_and(mbar_wait(smem_u32(mbar), (s - s_begin) & 1u)) != 0;
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        if (!ok) break;
        // ---- epilogue: ||q_s||^2 + ||c||^2 - 2 q.c, clamped at 0
        float qn = 0.0f;
        for (uint32_t j = o; j < o + ds; ++j) {
            const float x = valid ? static_cast<float>(qp[j]) : 0.0f;
            qn = __fmaf_rn(x, x, qn);
        }
        const uint64_t row = static_cast<uint64_t>(valid ? q : 0u) * a.M * kN + static_cast<uint64_t>(s) * kN;
        for (uint32_t c0 = 0; c0 < kN; c0 += 32) {
            float v[32];
            tmem_ld32(tmem + ((warp * 32u) << 16) + c0, v);
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                float x = __fadd_rn(__fadd_rn(qn, cn[c0 + i]), -2.0f * v[i]);
                v[i] = x > 0.0f ? x : 0.0f;
            }
            if (valid) {
                if (a.out_bf16) {
                    uint32_t w[16];
#pragma unroll
                    for (int i = 0; i < 16; ++i)
                        w[i] = static_cast<uint32_t>(__bfloat16_as_ushort(__float2bfloat16_rn(v[2 * i]))) |
                               (static_cast<uint32_t>(__bfloat16_as_ushort(__float2bfloat16_rn(v[2 * i + 1]))) << 16);
                    uint4 *out = reinterpret_cast<uint4 *>(static_cast<uint16_t *>(a.out) + row + c0);
#pragma unroll
                    for (int i = 0; i < 4; ++i) out[i] = make_uint4(w[4 * i], w[4 * i + 1], w[4 * i + 2], w[4 * i + 3]);
                } else {
                    float4 *out = reinterpret_cast<float4 *>(static_cast<float *>(a.out) + row + c0);
#pragma unroll
                    for (int i = 0; i < 8; ++i) out[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
                }
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        __syncthreads();                               // TMEM and B buffer free for the next subspace
    }
    if (!ok && t == 0) atomicExch(a.err, 1u);
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kN) : "memory");
    }
}

}  // namespace

uint32_t tc_table_smem_bytes(uint32_t d, int dtype)
{
    (void)d;
    (void)dtype;
    return 3u * kMaxKbPerSub * kACore + 3u * kMaxKbPerSub * kBCore + kN * 4u + 16u;
}

cudaError_t launch_tc_tables(const TcTableArgs &a, int dtype, cudaStream_t st)
{
    const uint32_t smem = tc_table_smem_bytes(a.d, dtype);
    const dim3 grid((a.nq + kTile - 1) / kTile, (a.M + kSubPerCta - 1) / kSubPerCta);
    cudaError_t e;
#define BANG_TC_LAUNCH(DT)                                                                          \
    e = cudaFuncSetAttribute(adc_table_tc_kernel<DT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem); \
    if (e != cudaSuccess) return e;                                                                 \
    adc_table_tc_kernel<DT><<<grid, 128, smem, st>>>(a)
    if (dtype == 0) { BANG_TC_LAUNCH(0); }
    else if (dtype == 1) { BANG_TC_LAUNCH(1); }
    else { BANG_TC_LAUNCH(2); }
#undef BANG_TC_LAUNCH
    return cudaGetLastError();
}

}  // namespace bang
