// Tensor-core PQ distance tables (see adc_table_tc.cu).
#pragma once

#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace bang {

constexpr uint32_t kMaxKbPerSub = 4;   // 16-wide K blocks one subspace may span

template <int DT> struct TcElem;
template <> struct TcElem<0> { using T = uint8_t; };
template <> struct TcElem<1> { using T = int8_t; };
template <> struct TcElem<2> { using T = float; };

struct TcTableArgs {
    const void *queries;        // device, nq*d elements
    uint32_t nq, d, M;
    const uint32_t *off;        // device, M+1 subspace offsets
    const unsigned char *btiles;// device, centroid tiles (hi, lo per K block) in core-matrix layout
    const uint32_t *bfirst;     // device, M: first tile of subspace s (in 8 KB tiles)
    const float *cnorm;         // device, M*256 squared centroid norms
    void *out;                  // device, nq*M*256 FP32 or BF16
    uint32_t out_bf16;
    uint32_t tf32;              // queries rounded to TF32 (pair with the TF32 centroid tiles)
    unsigned int *err;          // device flag, set to 1 if a wait gave up
};

uint32_t tc_table_smem_bytes(uint32_t d, int dtype);
cudaError_t launch_tc_tables(const TcTableArgs &a, int dtype, cudaStream_t st);

}  // namespace bang
