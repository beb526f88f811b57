// Stage kernels with f64 storage (instantiations of stage_impl.cuh).
#include "stage_impl.cuh"

namespace dwf {
template void launch_stage_prec<TF64>(StageMode, bool, const StageArgs &, cudaStream_t);
}  // namespace dwf
