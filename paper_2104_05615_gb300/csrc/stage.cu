// Stage launch dispatch by storage precision, and the launch-shape fit test
// used by the autotuner (kernels: stage_impl.cuh, instantiated per precision
// in stage_f64.cu, stage_f32.cu, stage_f16.cu, stage_bf16.cu).
#include "stage_tc.cuh"

namespace dwf {

extern template void launch_stage_prec<TF64>(StageMode, bool, const StageArgs &, cudaStream_t);
extern template void launch_stage_prec<TF32>(StageMode, bool, const StageArgs &, cudaStream_t);
extern template void launch_stage_prec<TF16>(StageMode, bool, const StageArgs &, cudaStream_t);
extern template void launch_stage_prec<TBF16>(StageMode, bool, const StageArgs &, cudaStream_t);
extern template void launch_stage_prec<TFX16>(StageMode, bool, const StageArgs &, cudaStream_t);
extern template void launch_stage_prec<TFX8>(StageMode, bool, const StageArgs &, cudaStream_t);
extern template void launch_stage_tc<TF16>(StageMode, bool, const StageArgs &, cudaStream_t);
extern template void launch_stage_tc<TBF16>(StageMode, bool, const StageArgs &, cudaStream_t);
extern template void launch_stage_tc<TFX16>(StageMode, bool, const StageArgs &, cudaStream_t);

void launch_stage(Prec prec, StageMode mode, bool mphi_in, const StageArgs &a, cudaStream_t st)
{
    if (a.nout == 0) return;
    if (a.gather == 2 && mode != MODE_5D) {
        // the hop on the tensor cores (16-bit storage)
        switch (prec) {
        case P16: launch_stage_tc<TF16>(mode, mphi_in, a, st); return;
        case PB16: launch_stage_tc<TBF16>(mode, mphi_in, a, st); return;
        case PFX16: launch_stage_tc<TFX16>(mode, mphi_in, a, st); return;
        default: throw std::runtime_error("tensor-core hop needs 16-bit storage");
        }
    }
    switch (prec) {
    case P64: launch_stage_prec<TF64>(mode, mphi_in, a, st); break;
    case P32: launch_stage_prec<TF32>(mode, mphi_in, a, st); break;
    case P16: launch_stage_prec<TF16>(mode, mphi_in, a, st); break;
    case PB16: launch_stage_prec<TBF16>(mode, mphi_in, a, st); break;
    case PFX16: launch_stage_prec<TFX16>(mode, mphi_in, a, st); break;
    case PFX8: launch_stage_prec<TFX8>(mode, mphi_in, a, st); break;
    }
}

bool stage_fits(Prec prec, int tile, int Ls, int gather)
{
    // the 8-bit format gathers directly (its 8-byte chunks have no bulk-copy
    // or tensor-core-hop instance)
    if (prec == PFX8 && gather != 0) return false;
    if (gather == 2) {
        // tensor-core hop: 16-bit storage, 8-site tiles, Ls in {4, 8, 12, 16}
        const bool half = prec == P16 || prec == PB16 || prec == PFX16;
        return half && tile == kTcSites && Ls % 4 == 0 && Ls >= 4 && Ls <= 16 &&
               tc_smem(Ls, true, true).total <= 220 * 1024 && kSegPad % tile == 0;
    }
    if (gather != 0 && gather != 1) return false;
    const int NC = prec == P64 ? 12 : prec == P32 ? 6 : 3;
    const int esz = prec == P64 ? 8 : prec == P32 ? 4 : 2;
    const int rsz = prec == P64 ? 8 : 4;
    const bool tc = prec == P16 || prec == PB16 || prec == PFX16 || prec == PFX8;
    const bool tma = gather == 1 && prec != P64;
    const StageSmem L = stage_smem(tile, Ls, NC, esz, rsz, tma, tc, scaled_format(prec) && Ls % 4 == 0, true, true);
    const int nthr = (tile * Ls + 31) / 32 * 32;
    // a tile never straddles two kSegPad-aligned segments
    return L.total <= 220 * 1024 && nthr <= 512 && tile > 0 && kSegPad % tile == 0 &&
           (!tc || (tile % 4 == 0 && Ls <= 16));  // tensor-core stages pair the n-tiles
}

}  // namespace dwf
