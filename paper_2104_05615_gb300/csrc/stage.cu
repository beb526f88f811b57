// Stage launch dispatch by storage precision, and the launch-shape fit test
// used by the autotuner (kernels: stage_impl.cuh, instantiated per precision
// in stage_f64.cu, stage_f32.cu, stage_f16.cu, stage_bf16.cu).
#include "stage_impl.cuh"

namespace dwf {

extern template void launch_stage_prec<TF64>(StageMode, bool, const StageArgs &, cudaStream_t);
extern template void launch_stage_prec<TF32>(StageMode, bool, const StageArgs &, cudaStream_t);
extern template void launch_stage_prec<TF16>(StageMode, bool, const StageArgs &, cudaStream_t);
extern template void launch_stage_prec<TBF16>(StageMode, bool, const StageArgs &, cudaStream_t);
extern template void launch_stage_prec<TFX16>(StageMode, bool, const StageArgs &, cudaStream_t);

void launch_stage(Prec prec, StageMode mode, bool mphi_in, const StageArgs &a, cudaStream_t st)
{
    if (a.nout == 0) return;
    switch (prec) {
    case P64: launch_stage_prec<TF64>(mode, mphi_in, a, st); break;
    case P32: launch_stage_prec<TF32>(mode, mphi_in, a, st); break;
    case P16: launch_stage_prec<TF16>(mode, mphi_in, a, st); break;
    case PB16: launch_stage_prec<TBF16>(mode, mphi_in, a, st); break;
    case PFX16: launch_stage_prec<TFX16>(mode, mphi_in, a, st); break;
    }
}

bool stage_fits(Prec prec, int tile, int Ls, int gather)
{
    const int NC = prec == P64 ? 12 : prec == P32 ? 6 : 3;
    const int esz = prec == P64 ? 8 : prec == P32 ? 4 : 2;
    const int rsz = prec == P64 ? 8 : 4;
    const bool tc = prec == P16 || prec == PB16 || prec == PFX16;
    const bool tma = gather == 1 && prec != P64;
    const StageSmem L = stage_smem(tile, Ls, NC, esz, rsz, tma, tc, scaled_format(prec) && Ls % 4 == 0, true, true);
    const int nthr = (tile * Ls + 31) / 32 * 32;
    // a tile never straddles two kSegPad-aligned segments
    return L.total <= 220 * 1024 && nthr <= 512 && tile > 0 && kSegPad % tile == 0 &&
           (!tc || (tile % 4 == 0 && Ls <= 16));  // tensor-core stages pair the n-tiles
}

}  // namespace dwf
