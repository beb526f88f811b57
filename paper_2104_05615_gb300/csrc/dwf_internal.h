// Internal declarations of the GB300 domain-wall library (not part of the ABI).
//
// Packed field layout (device): sites in block-major order (all sites of
// block 0, then block 1, ...; block-local lexicographic order inside a block,
// padded to a multiple of kSegPad sites); inside a site, 16-byte chunks of the
// 24 reals of a 5D site are laid out as [site][chunk][s][16 bytes], so a warp
// whose lanes run over s reads contiguous 16-byte words.  FP16 fields carry
// one FP32 scale per (site, s) colour-spinor, [site][s].
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <stdexcept>
#include <string>
#include <vector>

#include "dwf.h"

namespace dwf {

enum Prec { P64 = 0, P32 = 1, P16 = 2, PB16 = 3, PFX16 = 4, PFX8 = 5 };
constexpr int kNumPrec = 6;
// formats stored with one FP32 scale per (site, s) after the data
inline bool scaled_format(Prec p) { return p == P16 || p == PFX16 || p == PFX8; }

constexpr int kSegPad = 32;  // every segment (block / system) is padded to this many sites

inline int elem_bytes(Prec p) { return p == P64 ? 8 : p == P32 ? 4 : p == PFX8 ? 1 : 2; }
inline size_t field_bytes(Prec p, long nsite, int Ls)
{
    size_t b = (size_t)nsite * Ls * 24 * elem_bytes(p);
    if (scaled_format(p)) b += (size_t)nsite * Ls * sizeof(float);
    return b;
}
// scale array of a scaled field sits right after its data
inline float *field_scale(void *data, Prec p, long nsite, int Ls)
{
    return scaled_format(p) ? (float *)((char *)data + (size_t)nsite * Ls * 24 * elem_bytes(p)) : nullptr;
}
inline const float *field_scale(const void *data, Prec p, long nsite, int Ls)
{
    return scaled_format(p) ? (const float *)((const char *)data + (size_t)nsite * Ls * 24 * elem_bytes(p))
                            : nullptr;
}

// One stage of an operator: out = Epilogue(F . hop(G . in)), see stage.cu.
enum StageMode { MODE_F = 0, MODE_S2 = 1, MODE_S4 = 2, MODE_5D = 3 };

struct StageArgs {
    const void *in;
    void *out;
    const int *nbr;      // [nout][8] input site index; -1 none; <= -2: index -e-2 with sign -1
    const void *links;   // [rows][8][12] first two rows of the link matrix applied to the neighbour
    const void *aux;     // MODE_S2: y = aux - F h; MODE_S4: out = G aux - F h
    const void *dotv;    // MODE_S4: partial <dotv, out> per CTA into dot_part
    double *dot_part;
    const void *F;       // [nsys][2][Ls][Ls] real, chirality 0 = spins 0,1
    const void *G;       // same, or null (identity)
    const uint16_t *tile_sys;  // system of every kSegPad-site output tile (null: system 0)
    const double *mphi;  // [nsys][5] = (b, c, mass, A, B): M_phi on load, S4 coefficients
    long nout;           // output sites (multiple of the CTA tile)
    long nin;            // input sites (for the FP16 scale offset)
    long naux;           // aux sites (for the FP16 scale offset)
    int Ls;
    int dagger;          // 1: (1 +- gamma) signs flipped (D^w^+)
    int tile;            // output sites per CTA
    int seg_out;         // output sites per segment (block)
    int link_stride;     // link rows per segment
    int aux_stride;      // aux sites per segment
    int aux_valid;       // aux present for local index < aux_valid
    int *err;            // device flag set when a bounded wait gives up (may be null)
    unsigned poll_limit; // polls of a bounded wait before it gives up (0: 2^22)
    int force_timeout;   // testing the failure path: after its copies have landed the
                         // CTA waits on a barrier phase that never completes
    int gather;          // 0: direct neighbour loads; 1: bulk-copy staging in shared memory
    const int *active;   // per system: 0 = converged, its CTAs exit at once (null: all active)
    long site0;          // first output site of this launch (a wave of blocks); indices stay absolute
    long site_end;       // one past the last output site of this launch (0: nout)
    int fprog;           // CUDA-core stages: FProg (structured fifth-dimension solve) or 0 (dense F, G)
};

// The fifth-dimension operators of a CUDA-core stage as structured solves
// (M5op = A + B P is bidiagonal up to one wrap term): FP_M5I M5^-1,
// FP_M5ID M5^-+, FP_S2 M5^-+ (aux - M5^-1 h).  FP_DENSE applies the dense F
// (and G).
enum FProg { FP_DENSE = 0, FP_M5I, FP_M5ID, FP_S2 };

// Does a (tile, gather) choice fit the per-CTA limits for this precision and Ls?
bool stage_fits(Prec prec, int tile, int Ls, int gather);

// Launch a stage kernel; prec selects storage (P64/P32/P16/PB16), mphi_in
// applies M_phi to every neighbour on load.
void launch_stage(Prec prec, StageMode mode, bool mphi_in, const StageArgs &a, cudaStream_t st);

// ---------------------------------------------------------------- BLAS
struct Seg {             // a partition of sites into segments of whole kSegPad tiles
    int nseg = 0;
    uint16_t *d_tile_seg = nullptr;   // [ntiles]
    int *d_tile_begin = nullptr;      // [nseg+1] first tile of each segment
    std::vector<int> h_tile_begin;
    long nsite = 0;
};

// Per-CTA partial sums use CTAs of `tile` sites x Ls threads.
void launch_convert(Prec pout, void *out, Prec pin, const void *in, long nsite, int Ls,
                    cudaStream_t st);
// canonical (complex, [s][cb][4][3]) <-> packed; perm[i] = canonical cb index of
// packed site i or -1 (padding)
void launch_pack(Prec p, void *packed, const void *canon, const long *perm, long nsite, long Vh,
                 int Ls, cudaStream_t st);
void launch_unpack(Prec p, void *canon, const void *packed, const long *perm, long nsite, long Vh,
                   int Ls, cudaStream_t st);

// Generic fused vector kernels over packed fields with per-segment scalars.
// See blas.cu for the exact formulas.
enum BlasOp {
    BLAS_DOT = 0,        // part <- sum <a, b>
    BLAS_NORM2,          // part <- |a|^2
    BLAS_CG_UPDATE,      // x += alpha p ; r -= alpha Ap ; part <- |r|^2
    BLAS_XPAY,           // p = r + beta p
    BLAS_AXPY_ZERO,      // a = 0
    BLAS_COPY,           // a = b (convert)
    BLAS_DOT2,           // part <- (<a,b>, <a,c>)
    BLAS_RESIDUAL,       // r = b - Ax (r FP64 / FP32 out) ; part <- |r|^2
};

struct BlasArgs {
    void *v[5];
    Prec p[5];
    const double *scal[2];   // per-segment scalars (alpha, beta)
    double scal_sign[2];
    const uint16_t *tile_seg;
    double *part;            // [nctas][2]
    long nsite;
    int Ls;
    int tile;
    const uint16_t *tile_sys;  // system of each kSegPad-site tile (with `active`)
    const int *active;         // per system: 0 = converged, skip (null: all active)
    long site0;                // first site of this launch; sites [site0, site_end) are processed
    long site_end;             // 0: nsite
    // BLAS_COPY / BLAS_XPAY: also write u = M_phi v (v the vector written to v[0]),
    // M_phi = -(b + c P)/2 per system (mphi = [nsys][5] = b, c, mass, ...)
    void *mphi_out;
    Prec mphi_prec;
    const double *mphi;
    // BLAS_CG_UPDATE: x_zero = x is zero on input (not read); v[4] (if set)
    // receives the updated x in precision p[4] instead of v[0]; v[2] null:
    // only the x half (no r update, no partial)
    int x_zero;
};
void launch_blas(BlasOp op, const BlasArgs &a, cudaStream_t st);

// Segment reductions of per-CTA partials and the CG scalar recurrences.
enum ScalarOp {
    SC_SUM = 0,          // out[s] = sum part
    SC_ALPHA,            // alpha = num / sum part   (num from buffer)
    SC_BETA_FR,          // beta = sum part / den ; den <- sum part
    SC_BETA_PR,          // beta = -alpha <z,Ap> / rz_old; rz <- <z,r>
};
struct ScalarArgs {
    const double *part;
    int ncomp;           // components per CTA partial (1 or 2)
    const int *tile_begin;  // [nseg+1]
    int nseg;
    int cta_tiles;       // kSegPad-tiles per CTA of the partial producer (fractional not allowed)
    int sites_per_cta;   // sites per CTA of the producer
    double *s0, *s1, *s2, *s3;  // op-specific scalar arrays [nseg]
    int seg0;            // first segment of this launch (nseg segments from seg0)
};
void launch_scalar(ScalarOp op, const ScalarArgs &a, cudaStream_t st);

// Fifth-dimension transform (reduced Ls): out[(s,a)] = sum T[(s,a),(t,b)] in[(t,b)]
// tensor_cores: BF16 operands with FP32 accumulation (for inner storage of
// BF16 precision or coarser; even Ls_in), else FP32 on the CUDA cores.
void launch_tapply(Prec pout, void *out, int Ls_out, Prec pin, const void *in, int Ls_in,
                   const float *T, long nsite, int dagger, const void *addv, Prec padd,
                   double add_coef, cudaStream_t st, bool tensor_cores = false);
// G (device, (4 La) x (4 Lb) complex) = sum over sites and colours of a b^+
// for canonical FP64 fields; work: tcontract_workspace_bytes(La, Lb) bytes.
size_t tcontract_workspace_bytes(int La, int Lb);
void launch_tcontract(double *G_dev, const double *a, int La, const double *b, int Lb, long Vh,
                      void *work, cudaStream_t st);

// Canonical complex fields of n elements (FP64 or FP32): out = a x + b y
// (y null: out = a x) and <a, b> into out_dev[2] (FP64, fixed-order sums;
// work: field_dot_workspace_bytes()).
void launch_field_axpby(void *out, Prec pout, const void *x, const void *y, Prec pin, double ar, double ai,
                        double br, double bi, long n, cudaStream_t st);
size_t field_dot_workspace_bytes();
void launch_field_dot(double *out_dev, const void *a, const void *b, Prec p, long n, void *work, cudaStream_t st);

// Process-wide launch counter (every launch_* adds its kernels).
void count_launch(long long n = 1);
long long launch_count();

// Errors
struct CudaError {
    cudaError_t err;
    const char *what;
};
#define DWF_CUDA(x)                                                             \
    do {                                                                        \
        cudaError_t e_ = (x);                                                   \
        if (e_ != cudaSuccess) throw ::dwf::CudaError{e_, #x};                  \
    } while (0)

}  // namespace dwf
