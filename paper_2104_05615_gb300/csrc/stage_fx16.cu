// Stage kernels for 16-bit fixed-point storage (int16 + FP32 scale per colour-spinor).
#include "stage_tc.cuh"

namespace dwf {
template void launch_stage_prec<TFX16>(StageMode, bool, const StageArgs &, cudaStream_t);
template void launch_stage_tc<TFX16>(StageMode, bool, const StageArgs &, cudaStream_t);
}  // namespace dwf
