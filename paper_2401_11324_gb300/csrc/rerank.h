// Staged re-rank kernel (§4.8), launched after a search that recorded its
// candidates (SearchArgs::cand).  Internal to the library.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace bang {

struct RerankArgs {
    const void *queries;      // device, nq rows of d elements
    const void *base;         // device-accessible vectors, row stride vstride elements
    uint32_t vstride, d;
    uint32_t vec_ok, vecb_ok; // rows of queries / base allow 4-element vector loads
    const uint32_t *cand;     // device, nq rows of cand_cap candidate ids
    uint32_t cand_cap;
    const uint32_t *cand_n;   // device, candidates per query
    uint32_t nq, k, L;        // k, L: the bounds; k is also the output row stride
    const uint32_t *k_per_q;  // device or null (batched form)
    const uint32_t *L_per_q;  // device or null
    uint32_t *out_ids;        // device, nq*k
    float *out_dist;          // device, nq*k
};

// dtype: 0 u8, 1 i8, 2 f32 (bang_dtype).
cudaError_t launch_rerank(const RerankArgs &a, int dtype, cudaStream_t st);

}  // namespace bang
