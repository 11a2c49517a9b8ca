// Instantiates the search kernel for one distance mode (see search_kernel.cuh).
#include "search_kernel.cuh"

namespace bang {
cudaError_t launch_search_f32lazy(const SearchArgs &a, int dtype, size_t smem, cudaStream_t st)
{
    return launch_mode<kModeF32Lazy>(a, dtype, smem, st);
}
}  // namespace bang
