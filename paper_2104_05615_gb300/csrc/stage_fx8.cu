// Stage kernels for 8-bit fixed-point storage (int8 + FP32 scale per colour-spinor).
#include "stage_impl.cuh"

namespace dwf {
template void launch_stage_prec<TFX8>(StageMode, bool, const StageArgs &, cudaStream_t);
}  // namespace dwf
