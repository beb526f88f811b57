// Stage kernels with f16 storage (instantiations of stage_impl.cuh).
#include "stage_tc.cuh"

namespace dwf {
template void launch_stage_prec<TF16>(StageMode, bool, const StageArgs &, cudaStream_t);
template void launch_stage_tc<TF16>(StageMode, bool, const StageArgs &, cudaStream_t);
}  // namespace dwf
