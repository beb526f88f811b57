// Stage kernels with f32 storage (instantiations of stage_impl.cuh).
#include "stage_impl.cuh"

namespace dwf {
template void launch_stage_prec<TF32>(StageMode, bool, const StageArgs &, cudaStream_t);
}  // namespace dwf
