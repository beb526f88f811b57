// Stage kernels with bf16 storage (instantiations of stage_impl.cuh).
#include "stage_tc.cuh"

namespace dwf {
template void launch_stage_prec<TBF16>(StageMode, bool, const StageArgs &, cudaStream_t);
template void launch_stage_tc<TBF16>(StageMode, bool, const StageArgs &, cudaStream_t);
}  // namespace dwf
