// Vector kernels of the Krylov solvers (Algorithm 1) over packed fields:
// fused axpy + norm updates, dot products with per-segment (per block or per
// system) partial sums, precision conversion, canonical <-> packed layout,
// the per-segment scalar recurrences of CG, and the reduced-Ls transform
// z = T^+ zhat + mu r of Sec. 3.3.
#include <algorithm>
#include <atomic>
#include <stdexcept>

#include "device_common.cuh"

namespace dwf {

static std::atomic<long long> g_launches{0};
void count_launch(long long n) { g_launches += n; }
long long launch_count() { return g_launches.load(); }

// ------------------------------------------------ precision-generic access
// kNo64: the caller never passes FP64 operands (blas_kernel<float>: launch_blas
// sends those to the double instance), so the FP64 branches are compiled out.
template <typename R, bool kNo64 = false>
__device__ __forceinline__ void load_any(Prec p, const void *base, long nsite, long site, int s,
                                         int Ls, R *v)
{
    switch (p) {
    case P64: {
        if constexpr (kNo64) break;
        double t[24];
        load_sp<TF64>(base, nsite, site, s, Ls, t);
#pragma unroll
        for (int r = 0; r < 24; r++) v[r] = (R)t[r];
    } break;
    case P32: {
        float t[24];
        load_sp<TF32>(base, nsite, site, s, Ls, t);
#pragma unroll
        for (int r = 0; r < 24; r++) v[r] = (R)t[r];
    } break;
    case P16: {
        float t[24];
        load_sp<TF16>(base, nsite, site, s, Ls, t);
#pragma unroll
        for (int r = 0; r < 24; r++) v[r] = (R)t[r];
    } break;
    case PFX16: {
        float t[24];
        load_sp<TFX16>(base, nsite, site, s, Ls, t);
#pragma unroll
        for (int r = 0; r < 24; r++) v[r] = (R)t[r];
    } break;
    case PFX8: {
        float t[24];
        load_sp<TFX8>(base, nsite, site, s, Ls, t);
#pragma unroll
        for (int r = 0; r < 24; r++) v[r] = (R)t[r];
    } break;
    default: {
        float t[24];
        load_sp<TBF16>(base, nsite, site, s, Ls, t);
#pragma unroll
        for (int r = 0; r < 24; r++) v[r] = (R)t[r];
    } break;
    }
}
template <typename R, bool kNo64 = false>
__device__ __forceinline__ void store_any(Prec p, void *base, long nsite, long site, int s,
                                          int Ls, const R *v)
{
    switch (p) {
    case P64: {
        if constexpr (kNo64) break;
        double t[24];
#pragma unroll
        for (int r = 0; r < 24; r++) t[r] = (double)v[r];
        store_sp<TF64>(base, nsite, site, s, Ls, t);
    } break;
    case P32: {
        float t[24];
#pragma unroll
        for (int r = 0; r < 24; r++) t[r] = (float)v[r];
        store_sp<TF32>(base, nsite, site, s, Ls, t);
    } break;
    case P16: {
        float t[24];
#pragma unroll
        for (int r = 0; r < 24; r++) t[r] = (float)v[r];
        store_sp<TF16>(base, nsite, site, s, Ls, t);
    } break;
    case PFX16: {
        float t[24];
#pragma unroll
        for (int r = 0; r < 24; r++) t[r] = (float)v[r];
        store_sp<TFX16>(base, nsite, site, s, Ls, t);
    } break;
    case PFX8: {
        float t[24];
#pragma unroll
        for (int r = 0; r < 24; r++) t[r] = (float)v[r];
        store_sp<TFX8>(base, nsite, site, s, Ls, t);
    } break;
    default: {
        float t[24];
#pragma unroll
        for (int r = 0; r < 24; r++) t[r] = (float)v[r];
        store_sp<TBF16>(base, nsite, site, s, Ls, t);
    } break;
    }
}

__device__ __forceinline__ void block_reduce_store(double v0, double v1, int ncomp, double *part,
                                                   long cta)
{
    __shared__ double red[2][32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v0 += __shfl_xor_sync(0xffffffffu, v0, o);
        v1 += __shfl_xor_sync(0xffffffffu, v1, o);
    }
    const int tid = threadIdx.x, nw = (blockDim.x + 31) / 32;
    if ((tid & 31) == 0) {
        red[0][tid >> 5] = v0;
        red[1][tid >> 5] = v1;
    }
    __syncthreads();
    if (tid < 32) {
        double a = tid < nw ? red[0][tid] : 0.0, b = tid < nw ? red[1][tid] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, o);
            b += __shfl_xor_sync(0xffffffffu, b, o);
        }
        if (tid == 0) {
            part[(size_t)cta * ncomp] = a;
            if (ncomp > 1) part[(size_t)cta * ncomp + 1] = b;
        }
    }
}

// One thread per 5D site (site, s); a CTA covers `tile` sites x Ls.  One
// instantiation per operation, so that each keeps only its own operands live:
// the single-precision instances stay within 64 registers (several CTAs per
// SM keep enough loads in flight for HBM).
template <typename R, int OP>
__global__ void __launch_bounds__(512, sizeof(R) == 4 ? 2 : 1) blas_kernel(BlasArgs a)
{
    const int Ls = a.Ls;
    const int jl = threadIdx.x / Ls, s = threadIdx.x - jl * Ls;
    const long i = a.site0 + (long)blockIdx.x * a.tile + jl;
    const long cta = a.site0 / a.tile + blockIdx.x;  // absolute CTA index (partials)
    const bool active = jl < a.tile && i < (a.site_end ? a.site_end : a.nsite);
    constexpr int ncomp = OP == BLAS_DOT2 ? 2 : 1;
    double p0 = 0, p1 = 0;
    const int seg = (active && a.tile_seg) ? a.tile_seg[i / kSegPad] : 0;
    const long n = a.nsite;
    if (a.active) {
        // converged systems of a batch are skipped (a CTA never straddles systems)
        const long i0 = a.site0 + (long)blockIdx.x * a.tile;
        const int sys = a.tile_sys ? a.tile_sys[i0 / kSegPad] : 0;
        if (!a.active[sys]) {
            if (a.part && threadIdx.x == 0)
                for (int c = 0; c < ncomp; c++) a.part[(size_t)cta * ncomp + c] = 0.0;
            return;
        }
    }
    if (active) {
        if constexpr (OP == BLAS_DOT || OP == BLAS_DOT2) {
            R v0[24];
            load_any<R, sizeof(R) == 4>(a.p[0], a.v[0], n, i, s, Ls, v0);
            {
                R v1[24];
                load_any<R, sizeof(R) == 4>(a.p[1], a.v[1], n, i, s, Ls, v1);
                R d = 0;
#pragma unroll
                for (int r = 0; r < 24; r++) d += v0[r] * v1[r];
                p0 = (double)d;
            }
            if constexpr (OP == BLAS_DOT2) {
                R v2[24];
                load_any<R, sizeof(R) == 4>(a.p[2], a.v[2], n, i, s, Ls, v2);
                R e = 0;
#pragma unroll
                for (int r = 0; r < 24; r++) e += v0[r] * v2[r];
                p1 = (double)e;
            }
        } else if constexpr (OP == BLAS_NORM2) {
            R v0[24];
            load_any<R, sizeof(R) == 4>(a.p[0], a.v[0], n, i, s, Ls, v0);
            R d = 0;
#pragma unroll
            for (int r = 0; r < 24; r++) d += v0[r] * v0[r];
            p0 = (double)d;
        } else if constexpr (OP == BLAS_CG_UPDATE) {
            // x += alpha p ; r -= alpha Ap ; |r|^2 (the two halves in turn)
            const R al = (R)(a.scal[0][seg] * a.scal_sign[0]);
            {
                R v0[24], v1[24];
                if (a.x_zero) {
#pragma unroll
                    for (int r = 0; r < 24; r++) v0[r] = 0;
                } else {
                    load_any<R, sizeof(R) == 4>(a.p[0], a.v[0], n, i, s, Ls, v0);
                }
                load_any<R, sizeof(R) == 4>(a.p[1], a.v[1], n, i, s, Ls, v1);
#pragma unroll
                for (int r = 0; r < 24; r++) v0[r] += al * v1[r];
                if (a.v[4]) store_any<R, sizeof(R) == 4>(a.p[4], a.v[4], n, i, s, Ls, v0);
                else store_any<R, sizeof(R) == 4>(a.p[0], a.v[0], n, i, s, Ls, v0);
            }
            if (a.v[2]) {
                R v2[24], v3[24];
                load_any<R, sizeof(R) == 4>(a.p[2], a.v[2], n, i, s, Ls, v2);
                load_any<R, sizeof(R) == 4>(a.p[3], a.v[3], n, i, s, Ls, v3);
                R d = 0;
#pragma unroll
                for (int r = 0; r < 24; r++) {
                    v2[r] -= al * v3[r];
                    d += v2[r] * v2[r];
                }
                store_any<R, sizeof(R) == 4>(a.p[2], a.v[2], n, i, s, Ls, v2);
                p0 = (double)d;
            }
        } else if constexpr (OP == BLAS_XPAY) {
            // v0 = v1 + beta v0
            const R be = (R)(a.scal[0][seg] * a.scal_sign[0]);
            R v0[24], v1[24];
            load_any<R, sizeof(R) == 4>(a.p[0], a.v[0], n, i, s, Ls, v0);
            load_any<R, sizeof(R) == 4>(a.p[1], a.v[1], n, i, s, Ls, v1);
#pragma unroll
            for (int r = 0; r < 24; r++) v0[r] = v1[r] + be * v0[r];
            store_any<R, sizeof(R) == 4>(a.p[0], a.v[0], n, i, s, Ls, v0);
        } else if constexpr (OP == BLAS_AXPY_ZERO) {
            R v0[24];
#pragma unroll
            for (int r = 0; r < 24; r++) v0[r] = 0;
            store_any<R, sizeof(R) == 4>(a.p[0], a.v[0], n, i, s, Ls, v0);
        } else if constexpr (OP == BLAS_COPY) {
            R v1[24];
            load_any<R, sizeof(R) == 4>(a.p[1], a.v[1], n, i, s, Ls, v1);
            store_any<R, sizeof(R) == 4>(a.p[0], a.v[0], n, i, s, Ls, v1);
            if (a.v[2]) store_any<R, sizeof(R) == 4>(a.p[2], a.v[2], n, i, s, Ls, v1);
            R d = 0;
#pragma unroll
            for (int r = 0; r < 24; r++) d += v1[r] * v1[r];
            p0 = (double)d;
        } else if constexpr (OP == BLAS_RESIDUAL) {
            // v0 = v1 - v2 ; optional copy into v3 ; |v0|^2
            R v1[24];
            load_any<R, sizeof(R) == 4>(a.p[1], a.v[1], n, i, s, Ls, v1);
            {
                R v2[24];
                load_any<R, sizeof(R) == 4>(a.p[2], a.v[2], n, i, s, Ls, v2);
#pragma unroll
                for (int r = 0; r < 24; r++) v1[r] -= v2[r];
            }
            R d = 0;
#pragma unroll
            for (int r = 0; r < 24; r++) d += v1[r] * v1[r];
            store_any<R, sizeof(R) == 4>(a.p[0], a.v[0], n, i, s, Ls, v1);
            if (a.v[3]) store_any<R, sizeof(R) == 4>(a.p[3], a.v[3], n, i, s, Ls, v1);
            p0 = (double)d;
        }
    }
    if constexpr (OP == BLAS_COPY || OP == BLAS_XPAY) {
        if (a.mphi_out) {
            // u = M_phi v for the vector just written (as stored): the CTA holds
            // whole Ls columns, so psi_{s+-1} of the same site come from shared
            // memory.  (M_phi v)_s = -(b v_s + c (P_- v_{s+1} + P_+ v_{s-1}))/2,
            // wrap terms times -mass.
            extern __shared__ __align__(16) unsigned char blas_smem[];
            R *sv = reinterpret_cast<R *>(blas_smem);
            R v[24];
            if (active) {
                load_any<R, sizeof(R) == 4>(a.p[0], a.v[0], n, i, s, Ls, v);
#pragma unroll
                for (int r = 0; r < 24; r++) sv[(jl * Ls + s) * 24 + r] = v[r];
            }
            __syncthreads();
            if (active) {
                const int sys = a.tile_sys ? a.tile_sys[i / kSegPad] : 0;
                const double *mp = a.mphi + 5 * sys;
                const R cb = (R)(-0.5 * mp[0]), cc = (R)(-0.5 * mp[1]), wm = (R)(-mp[2]);
                const int sp = s + 1 < Ls ? s + 1 : 0, sm = s > 0 ? s - 1 : Ls - 1;
                const R fp = s + 1 < Ls ? cc : cc * wm, fm = s > 0 ? cc : cc * wm;
                const R *vp = sv + (jl * Ls + sp) * 24, *vm = sv + (jl * Ls + sm) * 24;
                R u[24];
#pragma unroll
                for (int r = 0; r < 12; r++) u[r] = cb * v[r] + fp * vp[r];
#pragma unroll
                for (int r = 12; r < 24; r++) u[r] = cb * v[r] + fm * vm[r];
                store_any<R, sizeof(R) == 4>(a.mphi_prec, a.mphi_out, n, i, s, Ls, u);
            }
        }
    }
    if (a.part) block_reduce_store(p0, p1, ncomp, a.part, cta);
}

template <typename R>
static void launch_blas_t(BlasOp op, const BlasArgs &a, unsigned nblk, int nthr, size_t sm, cudaStream_t st)
{
    switch (op) {
    case BLAS_DOT: blas_kernel<R, BLAS_DOT><<<nblk, nthr, sm, st>>>(a); break;
    case BLAS_NORM2: blas_kernel<R, BLAS_NORM2><<<nblk, nthr, sm, st>>>(a); break;
    case BLAS_CG_UPDATE: blas_kernel<R, BLAS_CG_UPDATE><<<nblk, nthr, sm, st>>>(a); break;
    case BLAS_XPAY: blas_kernel<R, BLAS_XPAY><<<nblk, nthr, sm, st>>>(a); break;
    case BLAS_AXPY_ZERO: blas_kernel<R, BLAS_AXPY_ZERO><<<nblk, nthr, sm, st>>>(a); break;
    case BLAS_COPY: blas_kernel<R, BLAS_COPY><<<nblk, nthr, sm, st>>>(a); break;
    case BLAS_DOT2: blas_kernel<R, BLAS_DOT2><<<nblk, nthr, sm, st>>>(a); break;
    case BLAS_RESIDUAL: blas_kernel<R, BLAS_RESIDUAL><<<nblk, nthr, sm, st>>>(a); break;
    }
}

// The same operations when every operand is FP32 (the outer iteration's
// vectors): each operand is streamed one 16-byte chunk at a time (six per 5D
// site), so only a few values are live per thread and more warps fit on an
// SM, keeping more loads in flight.
__device__ __forceinline__ float4 ld4(const void *base, long site, int c, int s, int Ls)
{
    return __ldg(reinterpret_cast<const float4 *>(base) + ((size_t)site * 6 + c) * Ls + s);
}
__device__ __forceinline__ void st4(void *base, long site, int c, int s, int Ls, float4 v)
{
    reinterpret_cast<float4 *>(base)[((size_t)site * 6 + c) * Ls + s] = v;
}
__device__ __forceinline__ float dot4(float4 x, float4 y) { return x.x * y.x + x.y * y.y + x.z * y.z + x.w * y.w; }
__device__ __forceinline__ float4 axpy4(float a, float4 x, float4 y)
{
    return make_float4(fmaf(a, x.x, y.x), fmaf(a, x.y, y.y), fmaf(a, x.z, y.z), fmaf(a, x.w, y.w));
}

template <int OP>
__global__ void __launch_bounds__(512, 3) blas32_kernel(BlasArgs a)
{
    const int Ls = a.Ls;
    const int jl = threadIdx.x / Ls, s = threadIdx.x - jl * Ls;
    const long i = a.site0 + (long)blockIdx.x * a.tile + jl;
    const long cta = a.site0 / a.tile + blockIdx.x;
    const bool active = jl < a.tile && i < (a.site_end ? a.site_end : a.nsite);
    constexpr int ncomp = OP == BLAS_DOT2 ? 2 : 1;
    const int seg = (active && a.tile_seg) ? a.tile_seg[i / kSegPad] : 0;
    if (a.active) {
        const long i0 = a.site0 + (long)blockIdx.x * a.tile;
        const int sys = a.tile_sys ? a.tile_sys[i0 / kSegPad] : 0;
        if (!a.active[sys]) {
            if (a.part && threadIdx.x == 0)
                for (int c = 0; c < ncomp; c++) a.part[(size_t)cta * ncomp + c] = 0.0;
            return;
        }
    }
    extern __shared__ __align__(16) unsigned char blas_smem[];
    float4 *sv = reinterpret_cast<float4 *>(blas_smem);  // [site][s][chunk] (M_phi output)
    float d0 = 0.f, d1 = 0.f;
    if (active) {
        if constexpr (OP == BLAS_DOT || OP == BLAS_DOT2) {
#pragma unroll
            for (int c = 0; c < 6; c++) {
                const float4 x = ld4(a.v[0], i, c, s, Ls);
                d0 += dot4(x, ld4(a.v[1], i, c, s, Ls));
                if constexpr (OP == BLAS_DOT2) d1 += dot4(x, ld4(a.v[2], i, c, s, Ls));
            }
        } else if constexpr (OP == BLAS_NORM2) {
#pragma unroll
            for (int c = 0; c < 6; c++) {
                const float4 x = ld4(a.v[0], i, c, s, Ls);
                d0 += dot4(x, x);
            }
        } else if constexpr (OP == BLAS_CG_UPDATE) {
            // x += alpha p ; r -= alpha Ap ; |r|^2
            const float al = (float)(a.scal[0][seg] * a.scal_sign[0]);
            void *xo = a.v[4] ? a.v[4] : a.v[0];
#pragma unroll
            for (int c = 0; c < 6; c++) {
                const float4 x = a.x_zero ? make_float4(0.f, 0.f, 0.f, 0.f) : ld4(a.v[0], i, c, s, Ls);
                st4(xo, i, c, s, Ls, axpy4(al, ld4(a.v[1], i, c, s, Ls), x));
            }
            if (a.v[2]) {
#pragma unroll
                for (int c = 0; c < 6; c++) {
                    const float4 r = axpy4(-al, ld4(a.v[3], i, c, s, Ls), ld4(a.v[2], i, c, s, Ls));
                    st4(a.v[2], i, c, s, Ls, r);
                    d0 += dot4(r, r);
                }
            }
        } else if constexpr (OP == BLAS_XPAY) {
            // v0 = v1 + beta v0
            const float be = (float)(a.scal[0][seg] * a.scal_sign[0]);
#pragma unroll
            for (int c = 0; c < 6; c++) {
                const float4 v = axpy4(be, ld4(a.v[0], i, c, s, Ls), ld4(a.v[1], i, c, s, Ls));
                st4(a.v[0], i, c, s, Ls, v);
                if (a.mphi_out) sv[(jl * Ls + s) * 6 + c] = v;
            }
        } else if constexpr (OP == BLAS_AXPY_ZERO) {
#pragma unroll
            for (int c = 0; c < 6; c++) st4(a.v[0], i, c, s, Ls, make_float4(0.f, 0.f, 0.f, 0.f));
        } else if constexpr (OP == BLAS_COPY) {
#pragma unroll
            for (int c = 0; c < 6; c++) {
                const float4 v = ld4(a.v[1], i, c, s, Ls);
                st4(a.v[0], i, c, s, Ls, v);
                if (a.v[2]) st4(a.v[2], i, c, s, Ls, v);
                if (a.mphi_out) sv[(jl * Ls + s) * 6 + c] = v;
                d0 += dot4(v, v);
            }
        }
    }
    if constexpr (OP == BLAS_COPY || OP == BLAS_XPAY) {
        if (a.mphi_out) {
            // u = M_phi v: (M_phi v)_s = -(b v_s + c (P_- v_{s+1} + P_+ v_{s-1}))/2,
            // wrap terms times -mass; chunks 0..2 hold spins 0, 1 (P_-), 3..5 spins 2, 3
            __syncthreads();
            if (active) {
                const int sys = a.tile_sys ? a.tile_sys[i / kSegPad] : 0;
                const double *mp = a.mphi + 5 * sys;
                const float cb = (float)(-0.5 * mp[0]), cc = (float)(-0.5 * mp[1]), wm = (float)(-mp[2]);
                const int sp = s + 1 < Ls ? s + 1 : 0, sm = s > 0 ? s - 1 : Ls - 1;
                const float fp = s + 1 < Ls ? cc : cc * wm, fm = s > 0 ? cc : cc * wm;
#pragma unroll
                for (int c = 0; c < 6; c++) {
                    const float4 v = sv[(jl * Ls + s) * 6 + c];
                    const float4 w = sv[(jl * Ls + (c < 3 ? sp : sm)) * 6 + c];
                    const float f = c < 3 ? fp : fm;
                    st4(a.mphi_out, i, c, s, Ls,
                        make_float4(cb * v.x + f * w.x, cb * v.y + f * w.y, cb * v.z + f * w.z, cb * v.w + f * w.w));
                }
            }
        }
    }
    if (a.part) block_reduce_store((double)d0, (double)d1, ncomp, a.part, cta);
}

template <int OP>
static void launch_b32(const BlasArgs &a, unsigned nblk, int nthr, size_t sm, cudaStream_t st)
{
    blas32_kernel<OP><<<nblk, nthr, sm, st>>>(a);
}

void launch_blas(BlasOp op, const BlasArgs &a, cudaStream_t st)
{
    if (a.nsite == 0) return;
    bool dbl = false, all32 = op != BLAS_RESIDUAL && (!a.mphi_out || a.mphi_prec == P32);
    for (int k = 0; k < 5; k++) {
        if (a.v[k] && a.p[k] == P64) dbl = true;
        if (a.v[k] && a.p[k] != P32) all32 = false;
    }
    const int nthr = a.tile * a.Ls;
    const long end = a.site_end ? a.site_end : a.nsite;
    const unsigned nblk = (unsigned)((end - a.site0 + a.tile - 1) / a.tile);
    const size_t sm = a.mphi_out ? (size_t)nthr * 24 * (dbl ? 8 : 4) : 0;
    if (all32) {
        switch (op) {
        case BLAS_DOT: launch_b32<BLAS_DOT>(a, nblk, nthr, sm, st); break;
        case BLAS_NORM2: launch_b32<BLAS_NORM2>(a, nblk, nthr, sm, st); break;
        case BLAS_CG_UPDATE: launch_b32<BLAS_CG_UPDATE>(a, nblk, nthr, sm, st); break;
        case BLAS_XPAY: launch_b32<BLAS_XPAY>(a, nblk, nthr, sm, st); break;
        case BLAS_AXPY_ZERO: launch_b32<BLAS_AXPY_ZERO>(a, nblk, nthr, sm, st); break;
        case BLAS_COPY: launch_b32<BLAS_COPY>(a, nblk, nthr, sm, st); break;
        case BLAS_DOT2: launch_b32<BLAS_DOT2>(a, nblk, nthr, sm, st); break;
        default: break;
        }
    } else if (dbl) {
        launch_blas_t<double>(op, a, nblk, nthr, sm, st);
    } else {
        launch_blas_t<float>(op, a, nblk, nthr, sm, st);
    }
    DWF_CUDA(cudaGetLastError());
    count_launch();
}

// x (FP64) += xacc (any) ; xacc = 0
__global__ void accum_kernel(void *x, const void *xacc_c, Prec pacc, long nsite, int Ls, int tile)
{
    const int jl = threadIdx.x / Ls, s = threadIdx.x - jl * Ls;
    const long i = (long)blockIdx.x * tile + jl;
    if (jl >= tile || i >= nsite) return;
    void *xacc = const_cast<void *>(xacc_c);
    double xv[24], av[24];
    load_any<double>(P64, x, nsite, i, s, Ls, xv);
    load_any<double>(pacc, xacc, nsite, i, s, Ls, av);
#pragma unroll
    for (int r = 0; r < 24; r++) {
        xv[r] += av[r];
        av[r] = 0;
    }
    store_any<double>(P64, x, nsite, i, s, Ls, xv);
    store_any<double>(pacc, xacc, nsite, i, s, Ls, av);
}

void launch_accum(void *x, void *xacc, Prec pacc, long nsite, int Ls, int tile, cudaStream_t st)
{
    accum_kernel<<<(unsigned)((nsite + tile - 1) / tile), tile * Ls, 0, st>>>(x, xacc, pacc, nsite,
                                                                                Ls, tile);
    DWF_CUDA(cudaGetLastError());
    count_launch();
}

// ------------------------------------------------------------- conversions
__global__ void convert_kernel(Prec pout, void *out, Prec pin, const void *in, long nsite, int Ls,
                               int tile)
{
    const int jl = threadIdx.x / Ls, s = threadIdx.x - jl * Ls;
    const long i = (long)blockIdx.x * tile + jl;
    if (jl >= tile || i >= nsite) return;
    if (pout == P64 || pin == P64) {
        double v[24];
        load_any<double>(pin, in, nsite, i, s, Ls, v);
        store_any<double>(pout, out, nsite, i, s, Ls, v);
    } else {
        float v[24];
        load_any<float>(pin, in, nsite, i, s, Ls, v);
        store_any<float>(pout, out, nsite, i, s, Ls, v);
    }
}

void launch_convert(Prec pout, void *out, Prec pin, const void *in, long nsite, int Ls,
                    cudaStream_t st)
{
    if (nsite == 0) return;
    const int tile = Ls <= 16 ? 16 : 8;
    convert_kernel<<<(unsigned)((nsite + tile - 1) / tile), tile * Ls, 0, st>>>(pout, out, pin, in,
                                                                                 nsite, Ls, tile);
    DWF_CUDA(cudaGetLastError());
    count_launch();
}

// canonical element (s, cb) -> 24 reals
template <typename R>
__device__ __forceinline__ void load_canon(Prec p, const void *base, long Vh, long cb, int s,
                                           R *v)
{
    const size_t off = ((size_t)s * Vh + cb) * 24;
    switch (p) {
    case P64: {
        const double *q = reinterpret_cast<const double *>(base) + off;
        for (int r = 0; r < 24; r++) v[r] = (R)q[r];
    } break;
    case P32:
    case PFX16:
    case PFX8: {  // fixed-point fields are exchanged as FP32
        const float *q = reinterpret_cast<const float *>(base) + off;
        for (int r = 0; r < 24; r++) v[r] = (R)q[r];
    } break;
    case P16: {
        const __half *q = reinterpret_cast<const __half *>(base) + off;
        for (int r = 0; r < 24; r++) v[r] = (R)__half2float(q[r]);
    } break;
    default: {
        const __nv_bfloat16 *q = reinterpret_cast<const __nv_bfloat16 *>(base) + off;
        for (int r = 0; r < 24; r++) v[r] = (R)__bfloat162float(q[r]);
    } break;
    }
}
template <typename R>
__device__ __forceinline__ void store_canon(Prec p, void *base, long Vh, long cb, int s,
                                            const R *v)
{
    const size_t off = ((size_t)s * Vh + cb) * 24;
    switch (p) {
    case P64: {
        double *q = reinterpret_cast<double *>(base) + off;
        for (int r = 0; r < 24; r++) q[r] = (double)v[r];
    } break;
    case P32:
    case PFX16:
    case PFX8: {
        float *q = reinterpret_cast<float *>(base) + off;
        for (int r = 0; r < 24; r++) q[r] = (float)v[r];
    } break;
    case P16: {
        __half *q = reinterpret_cast<__half *>(base) + off;
        for (int r = 0; r < 24; r++) q[r] = __float2half_rn((float)v[r]);
    } break;
    default: {
        __nv_bfloat16 *q = reinterpret_cast<__nv_bfloat16 *>(base) + off;
        for (int r = 0; r < 24; r++) q[r] = __float2bfloat16_rn((float)v[r]);
    } break;
    }
}

__global__ void pack_kernel(Prec p, void *packed, const void *canon, const long *perm, long nsite,
                            long Vh, int Ls, int tile, int unpack)
{
    const int jl = threadIdx.x / Ls, s = threadIdx.x - jl * Ls;
    const long i = (long)blockIdx.x * tile + jl;
    if (jl >= tile || i >= nsite) return;
    const long cb = perm[i];
    if (p == P64) {
        double v[24];
        if (!unpack) {
            if (cb >= 0) load_canon<double>(p, canon, Vh, cb, s, v);
            else for (int r = 0; r < 24; r++) v[r] = 0;
            store_any<double>(p, packed, nsite, i, s, Ls, v);
        } else if (cb >= 0) {
            load_any<double>(p, packed, nsite, i, s, Ls, v);
            store_canon<double>(p, const_cast<void *>(canon), Vh, cb, s, v);
        }
    } else {
        float v[24];
        if (!unpack) {
            if (cb >= 0) load_canon<float>(p, canon, Vh, cb, s, v);
            else for (int r = 0; r < 24; r++) v[r] = 0;
            store_any<float>(p, packed, nsite, i, s, Ls, v);
        } else if (cb >= 0) {
            load_any<float>(p, packed, nsite, i, s, Ls, v);
            store_canon<float>(p, const_cast<void *>(canon), Vh, cb, s, v);
        }
    }
}

void launch_pack(Prec p, void *packed, const void *canon, const long *perm, long nsite, long Vh,
                 int Ls, cudaStream_t st)
{
    const int tile = Ls <= 16 ? 16 : 8;
    pack_kernel<<<(unsigned)((nsite + tile - 1) / tile), tile * Ls, 0, st>>>(p, packed, canon, perm,
                                                                              nsite, Vh, Ls, tile, 0);
    DWF_CUDA(cudaGetLastError());
    count_launch();
}
void launch_unpack(Prec p, void *canon, const void *packed, const long *perm, long nsite, long Vh,
                   int Ls, cudaStream_t st)
{
    const int tile = Ls <= 16 ? 16 : 8;
    pack_kernel<<<(unsigned)((nsite + tile - 1) / tile), tile * Ls, 0, st>>>(
        p, const_cast<void *>(packed), canon, perm, nsite, Vh, Ls, tile, 1);
    DWF_CUDA(cudaGetLastError());
    count_launch();
}

// ------------------------------------------------------------ scalars
// One CTA per segment sums the per-CTA partials of its sites, then thread 0
// applies the recurrence.
__global__ void scalar_kernel(ScalarOp op, ScalarArgs a)
{
    const int seg = a.seg0 + blockIdx.x;
    const long c0 = (long)a.tile_begin[seg] * kSegPad / a.sites_per_cta;
    const long c1 = (long)a.tile_begin[seg + 1] * kSegPad / a.sites_per_cta;
    double v0 = 0, v1 = 0;
    for (long c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
        v0 += a.part[c * a.ncomp];
        if (a.ncomp > 1) v1 += a.part[c * a.ncomp + 1];
    }
    __shared__ double red[2][32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v0 += __shfl_xor_sync(0xffffffffu, v0, o);
        v1 += __shfl_xor_sync(0xffffffffu, v1, o);
    }
    const int tid = threadIdx.x, nw = blockDim.x / 32;
    if ((tid & 31) == 0) {
        red[0][tid >> 5] = v0;
        red[1][tid >> 5] = v1;
    }
    __syncthreads();
    if (tid == 0) {
        double t0 = 0, t1 = 0;
        for (int w = 0; w < nw; w++) {
            t0 += red[0][w];
            t1 += red[1][w];
        }
        switch (op) {
        case SC_SUM:
            a.s0[seg] = t0;
            if (a.s1) a.s1[seg] = t1;
            break;
        case SC_ALPHA: {
            // alpha = num / <p, Ap>; an exact zero stops the segment
            const double num = a.s0[seg];
            a.s1[seg] = (num != 0.0 && t0 != 0.0) ? num / t0 : 0.0;
            if (a.s2) a.s2[seg] = t0;
        } break;
        case SC_BETA_FR: {
            const double old = a.s0[seg];
            a.s1[seg] = old != 0.0 ? t0 / old : 0.0;
            a.s0[seg] = t0;
            if (a.s2) a.s2[seg] = t0;
        } break;
        case SC_BETA_PR: {
            // beta = <z_new, r_new - r_old> / <z_old, r_old> with r_new - r_old = -alpha Ap
            const double old = a.s0[seg], al = a.s1[seg];
            a.s2[seg] = old != 0.0 ? -al * t1 / old : 0.0;
            a.s0[seg] = t0;
        } break;
        }
    }
}

void launch_scalar(ScalarOp op, const ScalarArgs &a, cudaStream_t st)
{
    scalar_kernel<<<a.nseg, 256, 0, st>>>(op, a);
    DWF_CUDA(cudaGetLastError());
    count_launch();
}

// ------------------------------------------------------ reduced-Ls transform
// out[(s,a)] = sum_{t,b} E[(s,a),(t,b)] in[(t,b)] per site and colour, with
// E = T (dagger = 0: Ls_in = 4 Ls columns of T, out at Ls_hat) or E = T^+
// (dagger = 1), then optionally out += add_coef * addv.  T complex float,
// (4 Ls_hat) x (4 Ls) row-major, as float pairs; arithmetic in FP32.
//
// Persistent CTAs: each stages E once, as [t][b][s][a] complex so that a
// thread's four output spins are contiguous, then walks tiles of sites: the
// tile's input columns go to shared memory and thread (site, s) accumulates
// its 4 spins x 3 colours, each input entry (t, b) read once and used for
// 48 fused multiply-adds.
constexpr int kTapplyThreads = 256;

__global__ void __launch_bounds__(kTapplyThreads) tapply_kernel(Prec pout, void *out, int Ls_out, Prec pin,
                                                                const void *in, int Ls_in, const float *T,
                                                                long nsite, int dagger, const void *addv,
                                                                Prec padd, double add_coef, int tile)
{
    extern __shared__ __align__(16) float sm_t[];
    float2 *sE = reinterpret_cast<float2 *>(sm_t);           // [4 Ls_in][Ls_out][4]
    float *sIn = sm_t + 2 * 16 * Ls_in * Ls_out;              // [tile][Ls_in][24]
    const int nin = 4 * Ls_in, nout = 4 * Ls_out;
    const int ncolT = dagger ? nout : nin;                    // columns of T (4 Ls)
    for (int e = threadIdx.x; e < nin * nout; e += blockDim.x) {
        const int tb = e / nout, sa = e - tb * nout;
        // E[(s,a),(t,b)]: T[sa][tb], or conj(T[tb][sa]) for T^+
        float2 v;
        if (!dagger) v = make_float2(T[2 * (sa * ncolT + tb)], T[2 * (sa * ncolT + tb) + 1]);
        else v = make_float2(T[2 * (tb * ncolT + sa)], -T[2 * (tb * ncolT + sa) + 1]);
        sE[e] = v;  // e = tb * nout + (s * 4 + a)
    }
    const int jl = threadIdx.x / Ls_out, s = threadIdx.x - jl * Ls_out;
    const long ntile = (nsite + tile - 1) / tile;
    for (long tl = blockIdx.x; tl < ntile; tl += gridDim.x) {
        __syncthreads();  // E staged / the previous tile's inputs consumed
        for (int e = threadIdx.x; e < tile * Ls_in; e += blockDim.x) {
            const int j = e / Ls_in, t = e - j * Ls_in;
            const long site = tl * tile + j;
            float v[24];
            if (site < nsite) load_any<float>(pin, in, nsite, site, t, Ls_in, v);
            else
#pragma unroll
                for (int r = 0; r < 24; r++) v[r] = 0.f;
            float4 *dst = reinterpret_cast<float4 *>(sIn + (j * Ls_in + t) * 24);
#pragma unroll
            for (int q = 0; q < 6; q++) dst[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
        }
        __syncthreads();
        const long i = tl * tile + jl;
        if (jl >= tile || i >= nsite) continue;
        float o[24];
#pragma unroll
        for (int r = 0; r < 24; r++) o[r] = 0.f;
        const float *x = sIn + jl * Ls_in * 24;
        for (int t = 0; t < Ls_in; t++) {
#pragma unroll
            for (int b = 0; b < 4; b++) {
                const float2 *xv = reinterpret_cast<const float2 *>(x + t * 24 + b * 6);
                const float2 x0 = xv[0], x1 = xv[1], x2 = xv[2];
                const float4 *ep = reinterpret_cast<const float4 *>(sE + ((t * 4 + b) * Ls_out + s) * 4);
                const float4 e01 = ep[0], e23 = ep[1];
                const float2 E[4] = {make_float2(e01.x, e01.y), make_float2(e01.z, e01.w),
                                     make_float2(e23.x, e23.y), make_float2(e23.z, e23.w)};
                const float2 X[3] = {x0, x1, x2};
#pragma unroll
                for (int a = 0; a < 4; a++)
#pragma unroll
                    for (int c = 0; c < 3; c++) {
                        float *oc = o + (a * 3 + c) * 2;
                        oc[0] = fmaf(E[a].x, X[c].x, fmaf(-E[a].y, X[c].y, oc[0]));
                        oc[1] = fmaf(E[a].x, X[c].y, fmaf(E[a].y, X[c].x, oc[1]));
                    }
            }
        }
        if (addv) {
            float w[24];
            load_any<float>(padd, addv, nsite, i, s, Ls_out, w);
#pragma unroll
            for (int r = 0; r < 24; r++) o[r] += (float)add_coef * w[r];
        }
        store_any<float>(pout, out, nsite, i, s, Ls_out, o);
    }
}

// Tensor-core form of the same transform, for an output stored in BF16
// precision or coarser (the forward map r -> T r into BF16 or 8-bit inner
// storage).  Per site and colour the map is a real product: rows (colour,
// site), K = (t, b, re/im) = 8 Ls_in, N = (s, a, re/im) = 8 Ls_out, with each
// complex E entry expanded to the real block [[Er, -Ei], [Ei, Er]].  BF16
// operands (the input rounded to the precision of the storage it feeds),
// FP32 accumulation, mma.sync m16n8k16.  Persistent CTAs of four warps stage
// the expanded E once as [n][k]; each tile of 16 sites is staged as the
// 48 x K operand [colour * 16 + site][k], multiplied (warp w takes n-tiles
// w, w + 4, ..., n-tile = output slice s), and written back per (site, s)
// through a shared FP32 buffer (the output formats with a scale per (site, s)
// need the whole colour-spinor).
constexpr int kTtcSites = 16;
constexpr int kTtcThreads = 128;

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint32_t pack_bf2(float lo, float hi)
{
    __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&h);
}
__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}
__device__ __forceinline__ void ldsm_x2(uint32_t addr, uint32_t &r0, uint32_t &r1)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];\n" : "=r"(r0), "=r"(r1) : "r"(addr));
}
__device__ __forceinline__ void mma_bf16_16816(float *d, uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                               uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// Shared memory of the tensor-core transform (bytes): E [N][K + 8] and the
// operand [48][K + 8] in BF16 (row pitch an odd number of 16-byte units for
// even Ls_in, so ldmatrix is conflict-free), the result [16][Ls_out][24] FP32.
__host__ __device__ inline size_t ttc_smem(int Ls_in, int Ls_out)
{
    const size_t kp = 8 * (size_t)Ls_in + 8;
    return 2 * kp * (8 * (size_t)Ls_out + 3 * kTtcSites) + 4 * (size_t)kTtcSites * Ls_out * 24;
}

__global__ void __launch_bounds__(kTtcThreads) tapply_tc_kernel(Prec pout, void *out, int Ls_out, Prec pin,
                                                                const void *in, int Ls_in, const float *T,
                                                                long nsite, int dagger, const void *addv,
                                                                Prec padd, double add_coef)
{
    extern __shared__ __align__(16) unsigned char sm_raw[];
    const int K = 8 * Ls_in, N = 8 * Ls_out, KP = K + 8;
    __nv_bfloat16 *sW = reinterpret_cast<__nv_bfloat16 *>(sm_raw);  // [N][KP]
    __nv_bfloat16 *sA = sW + (size_t)N * KP;                            // [48][KP]
    float *sC = reinterpret_cast<float *>(sA + (size_t)3 * kTtcSites * KP);  // [16][Ls_out][24]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int ncolT = 4 * (dagger ? Ls_out : Ls_in);  // columns of T (4 Ls)
    for (int e = tid; e < N * K; e += kTtcThreads) {
        const int n = e / K, k = e - n * K;
        const int sa = n >> 1, ro = n & 1, tb = k >> 1, ri = k & 1;
        // E[(s,a),(t,b)]: T[sa][tb], or conj(T[tb][sa]) for T^+
        float er, ei;
        if (!dagger) {
            er = T[2 * (sa * ncolT + tb)];
            ei = T[2 * (sa * ncolT + tb) + 1];
        } else {
            er = T[2 * (tb * ncolT + sa)];
            ei = -T[2 * (tb * ncolT + sa) + 1];
        }
        const float w = ro == 0 ? (ri == 0 ? er : -ei) : (ri == 0 ? ei : er);
        sW[(size_t)n * KP + k] = __float2bfloat16_rn(w);
    }
    const int g = lane >> 2, tg = lane & 3;
    const long ntile = (nsite + kTtcSites - 1) / kTtcSites;
    for (long tl = blockIdx.x; tl < ntile; tl += gridDim.x) {
        __syncthreads();  // E staged / the previous tile's operand and result consumed
        // operand rows (colour c, site j), k = (t * 4 + b) * 2 + re/im
        for (int e = tid; e < kTtcSites * Ls_in; e += kTtcThreads) {
            const int j = e / Ls_in, t = e - j * Ls_in;
            const long site = tl * kTtcSites + j;
            float v[24];
            if (site < nsite) load_any<float>(pin, in, nsite, site, t, Ls_in, v);
            else
#pragma unroll
                for (int r = 0; r < 24; r++) v[r] = 0.f;
#pragma unroll
            for (int q = 0; q < 12; q++) {  // component pair q = b * 3 + c: (re, im)
                const int b = q / 3, c = q - 3 * b;
                *reinterpret_cast<uint32_t *>(sA + (size_t)(c * kTtcSites + j) * KP + (t * 4 + b) * 2) =
                    pack_bf2(v[2 * q], v[2 * q + 1]);
            }
        }
        __syncthreads();
        for (int nt = warp; nt < Ls_out; nt += kTtcThreads / 32) {
#pragma unroll
            for (int c = 0; c < 3; c++) {
                float d[4] = {0.f, 0.f, 0.f, 0.f};
                for (int ks = 0; ks < K; ks += 16) {
                    uint32_t a0, a1, a2, a3, b0, b1;
                    const __nv_bfloat16 *pb = sW + (size_t)(nt * 8 + (lane & 7)) * KP + ks + 8 * ((lane >> 3) & 1);
                    ldsm_x2(smem_addr(pb), b0, b1);
                    const __nv_bfloat16 *pa =
                        sA + (size_t)(c * kTtcSites + (lane & 7) + 8 * ((lane >> 3) & 1)) * KP + ks + 8 * (lane >> 4);
                    ldsm_x4(smem_addr(pa), a0, a1, a2, a3);
                    mma_bf16_16816(d, a0, a1, a2, a3, b0, b1);
                }
                // rows g, g + 8 = sites; columns 2 tg, 2 tg + 1 = (s = nt, a = tg, re / im)
                float2 *c0 = reinterpret_cast<float2 *>(sC + ((size_t)g * Ls_out + nt) * 24 + (tg * 3 + c) * 2);
                float2 *c1 = reinterpret_cast<float2 *>(sC + ((size_t)(g + 8) * Ls_out + nt) * 24 + (tg * 3 + c) * 2);
                *c0 = make_float2(d[0], d[1]);
                *c1 = make_float2(d[2], d[3]);
            }
        }
        __syncthreads();
        for (int e = tid; e < kTtcSites * Ls_out; e += kTtcThreads) {
            const int j = e / Ls_out, s = e - j * Ls_out;
            const long site = tl * kTtcSites + j;
            if (site >= nsite) continue;
            float o[24];
            const float4 *src = reinterpret_cast<const float4 *>(sC + (size_t)e * 24);
#pragma unroll
            for (int q = 0; q < 6; q++) {
                const float4 f = src[q];
                o[4 * q] = f.x;
                o[4 * q + 1] = f.y;
                o[4 * q + 2] = f.z;
                o[4 * q + 3] = f.w;
            }
            if (addv) {
                float w[24];
                load_any<float>(padd, addv, nsite, site, s, Ls_out, w);
#pragma unroll
                for (int r = 0; r < 24; r++) o[r] += (float)add_coef * w[r];
            }
            store_any<float>(pout, out, nsite, site, s, Ls_out, o);
        }
    }
}

static bool launch_tapply_tc(Prec pout, void *out, int Ls_out, Prec pin, const void *in, int Ls_in,
                             const float *T, long nsite, int dagger, const void *addv, Prec padd,
                             double add_coef, cudaStream_t st)
{
    // K = 8 Ls_in must be a whole number of 16-wide k-steps
    // outputs of BF16 precision or coarser only
    if (pout != PB16 && pout != PFX8) return false;
    if (Ls_in % 2 != 0 || Ls_in > 16 || Ls_out > 16) return false;
    const size_t smem = ttc_smem(Ls_in, Ls_out);
    static bool attr = false;
    if (!attr) {
        DWF_CUDA(cudaFuncSetAttribute(tapply_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
        attr = true;
    }
    int dev = 0, nsm = 0, per_sm = 0;
    DWF_CUDA(cudaGetDevice(&dev));
    DWF_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    DWF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tapply_tc_kernel, kTtcThreads, smem));
    const long ntile = (nsite + kTtcSites - 1) / kTtcSites;
    const unsigned grid = (unsigned)std::max<long>(1, std::min<long>(ntile, (long)nsm * std::max(1, per_sm)));
    tapply_tc_kernel<<<grid, kTtcThreads, smem, st>>>(pout, out, Ls_out, pin, in, Ls_in, T, nsite, dagger, addv,
                                                       padd, add_coef);
    DWF_CUDA(cudaGetLastError());
    count_launch();
    return true;
}

void launch_tapply(Prec pout, void *out, int Ls_out, Prec pin, const void *in, int Ls_in,
                   const float *T, long nsite, int dagger, const void *addv, Prec padd,
                   double add_coef, cudaStream_t st, bool tensor_cores)
{
    if (nsite == 0) return;
    if (tensor_cores &&
        launch_tapply_tc(pout, out, Ls_out, pin, in, Ls_in, T, nsite, dagger, addv, padd, add_coef, st))
        return;
    const int tile = std::max(1, kTapplyThreads / Ls_out);
    const size_t smem = sizeof(float) * (2 * 16 * (size_t)Ls_out * Ls_in + (size_t)tile * Ls_in * 24);
    static bool attr = false;
    if (!attr) {
        DWF_CUDA(cudaFuncSetAttribute(tapply_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      200 * 1024));
        attr = true;
    }
    if (smem > 200 * 1024) throw std::runtime_error("reduced-Ls transform: fifth extents too large");
    int dev = 0, nsm = 0, per_sm = 0;
    DWF_CUDA(cudaGetDevice(&dev));
    DWF_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    DWF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tapply_kernel, tile * Ls_out, smem));
    const long ntile = (nsite + tile - 1) / tile;
    const unsigned grid = (unsigned)std::max<long>(1, std::min<long>(ntile, (long)nsm * std::max(1, per_sm)));
    tapply_kernel<<<grid, tile * Ls_out, smem, st>>>(pout, out, Ls_out, pin, in, Ls_in, T, nsite, dagger, addv,
                                                    padd, add_coef, tile);
    DWF_CUDA(cudaGetLastError());
    count_launch();
}

// ------------------------------------------------ transform contraction
// G[(s*4+mu)][(t*4+nu)] = sum over sites x and colours c of
//   a[s][x][mu][c] * conj(b[t][x][nu][c])
// for canonical FP64 fields a (La slices) and b (Lb slices): the outer
// products that make the gradient of the reduced-Ls loss (Sec. 3.3).  A fixed
// grid of CTAs strides over chunks of sites, each writing its partial matrix;
// a second kernel sums the partials in a fixed order (deterministic).
constexpr int kContractCtas = 304, kContractSites = 8, kContractThreads = 256, kContractMaxP = 16;

__global__ void __launch_bounds__(kContractThreads) tcontract_kernel(const double2 *a, int La,
                                                                      const double2 *b, int Lb, long Vh,
                                                                      double2 *part)
{
    extern __shared__ __align__(16) double2 sm_c[];
    const int na = La * 12, nb = Lb * 12, npair = 16 * La * Lb, ncol = 4 * Lb;
    double2 *sa = sm_c, *sb = sm_c + kContractSites * na;
    double ar[kContractMaxP], ai[kContractMaxP];
#pragma unroll
    for (int k = 0; k < kContractMaxP; k++) ar[k] = ai[k] = 0.0;
    const int tid = threadIdx.x;
    for (long x0 = (long)blockIdx.x * kContractSites; x0 < Vh; x0 += (long)gridDim.x * kContractSites) {
        for (int e = tid; e < kContractSites * na; e += kContractThreads) {
            const int j = e / na, q = e - j * na, sl = q / 12, rest = q - sl * 12;
            const long x = x0 + j;
            sa[e] = x < Vh ? a[((long)sl * Vh + x) * 12 + rest] : make_double2(0.0, 0.0);
        }
        for (int e = tid; e < kContractSites * nb; e += kContractThreads) {
            const int j = e / nb, q = e - j * nb, sl = q / 12, rest = q - sl * 12;
            const long x = x0 + j;
            sb[e] = x < Vh ? b[((long)sl * Vh + x) * 12 + rest] : make_double2(0.0, 0.0);
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kContractMaxP; k++) {
            const int pr = tid + k * kContractThreads;
            if (pr >= npair) break;
            const int row = pr / ncol, col = pr - row * ncol;
            const int oa = (row >> 2) * 12 + (row & 3) * 3, ob = (col >> 2) * 12 + (col & 3) * 3;
            double rr = ar[k], ii = ai[k];
            for (int j = 0; j < kContractSites; j++)
#pragma unroll
                for (int c = 0; c < 3; c++) {
                    const double2 u = sa[j * na + oa + c], v = sb[j * nb + ob + c];
                    rr += u.x * v.x + u.y * v.y;   // u conj(v)
                    ii += u.y * v.x - u.x * v.y;
                }
            ar[k] = rr;
            ai[k] = ii;
        }
        __syncthreads();
    }
#pragma unroll
    for (int k = 0; k < kContractMaxP; k++) {
        const int pr = tid + k * kContractThreads;
        if (pr < npair) part[(size_t)blockIdx.x * npair + pr] = make_double2(ar[k], ai[k]);
    }
}

__global__ void tcontract_reduce(const double2 *part, int nctas, int npair, double2 *G)
{
    const int pr = blockIdx.x * blockDim.x + threadIdx.x;
    if (pr >= npair) return;
    double2 s = make_double2(0.0, 0.0);
    for (int k = 0; k < nctas; k++) {
        const double2 v = part[(size_t)k * npair + pr];
        s.x += v.x;
        s.y += v.y;
    }
    G[pr] = s;
}

size_t tcontract_workspace_bytes(int La, int Lb)
{
    return (size_t)(kContractCtas + 1) * 16 * La * Lb * sizeof(double2);
}

void launch_tcontract(double *G_dev, const double *a, int La, const double *b, int Lb, long Vh,
                      void *work, cudaStream_t st)
{
    if (La < 1 || Lb < 1 || La * Lb > kContractThreads * kContractMaxP / 16)
        throw std::runtime_error("transform contraction: 16 La Lb must not exceed 4096");
    const int npair = 16 * La * Lb;
    const size_t smem = (size_t)kContractSites * 12 * (La + Lb) * sizeof(double2);
    static bool attr = false;
    if (!attr) {
        DWF_CUDA(cudaFuncSetAttribute(tcontract_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      200 * 1024));
        attr = true;
    }
    double2 *part = reinterpret_cast<double2 *>(work);
    tcontract_kernel<<<kContractCtas, kContractThreads, smem, st>>>(
        reinterpret_cast<const double2 *>(a), La, reinterpret_cast<const double2 *>(b), Lb, Vh, part);
    DWF_CUDA(cudaGetLastError());
    tcontract_reduce<<<(npair + 255) / 256, 256, 0, st>>>(part, kContractCtas, npair,
                                                          reinterpret_cast<double2 *>(G_dev));
    DWF_CUDA(cudaGetLastError());
    count_launch(2);
}

}  // namespace dwf

namespace dwf {

// ------------------------------------------- canonical-field axpby and dot
// out = a x + b y on canonical complex fields of n elements (x, y in pin,
// out in pout: FP64 or FP32 complex); y null: out = a x (a cast for a = 1).
template <typename TO, typename TI>
__global__ void field_axpby_kernel(TO *out, const TI *x, const TI *y, double ar, double ai, double br, double bi,
                                   long n)
{
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
        const double xr = (double)x[2 * e], xi = (double)x[2 * e + 1];
        double r = ar * xr - ai * xi, i = ar * xi + ai * xr;
        if (y) {
            const double yr = (double)y[2 * e], yi = (double)y[2 * e + 1];
            r += br * yr - bi * yi;
            i += br * yi + bi * yr;
        }
        out[2 * e] = (TO)r;
        out[2 * e + 1] = (TO)i;
    }
}

void launch_field_axpby(void *out, Prec pout, const void *x, const void *y, Prec pin, double ar, double ai,
                        double br, double bi, long n, cudaStream_t st)
{
    const int nthr = 256;
    const unsigned nblk = (unsigned)std::min<long>((n + nthr - 1) / nthr, 152L * 16);
    if (nblk == 0) return;
    if (pout == P64 && pin == P64)
        field_axpby_kernel<double, double><<<nblk, nthr, 0, st>>>((double *)out, (const double *)x,
                                                                 (const double *)y, ar, ai, br, bi, n);
    else if (pout == P64)
        field_axpby_kernel<double, float><<<nblk, nthr, 0, st>>>((double *)out, (const float *)x,
                                                                (const float *)y, ar, ai, br, bi, n);
    else if (pin == P64)
        field_axpby_kernel<float, double><<<nblk, nthr, 0, st>>>((float *)out, (const double *)x,
                                                                (const double *)y, ar, ai, br, bi, n);
    else
        field_axpby_kernel<float, float><<<nblk, nthr, 0, st>>>((float *)out, (const float *)x,
                                                               (const float *)y, ar, ai, br, bi, n);
    DWF_CUDA(cudaGetLastError());
    count_launch();
}

// <a, b> = sum conj(a_e) b_e in FP64: a fixed grid of CTAs, each thread a
// fixed stride of elements, per-CTA partials summed by one CTA in a fixed
// order, so the result does not depend on scheduling.
constexpr int kDotCtas = 304, kDotThreads = 256;

template <typename TI>
__global__ void __launch_bounds__(kDotThreads) field_dot_kernel(const TI *a, const TI *b, long n, double2 *part)
{
    double r = 0.0, i = 0.0;
    for (long e = (long)blockIdx.x * kDotThreads + threadIdx.x; e < n; e += (long)kDotCtas * kDotThreads) {
        const double ar = (double)a[2 * e], ai = (double)a[2 * e + 1];
        const double br = (double)b[2 * e], bi = (double)b[2 * e + 1];
        r += ar * br + ai * bi;
        i += ar * bi - ai * br;
    }
    __shared__ double sr[kDotThreads], si[kDotThreads];
    sr[threadIdx.x] = r;
    si[threadIdx.x] = i;
    __syncthreads();
    for (int o = kDotThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            sr[threadIdx.x] += sr[threadIdx.x + o];
            si[threadIdx.x] += si[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = make_double2(sr[0], si[0]);
}

__global__ void field_dot_reduce(const double2 *part, double2 *out)
{
    if (threadIdx.x != 0) return;
    double r = 0.0, i = 0.0;
    for (int k = 0; k < kDotCtas; k++) {
        r += part[k].x;
        i += part[k].y;
    }
    *out = make_double2(r, i);
}

size_t field_dot_workspace_bytes() { return (kDotCtas + 1) * sizeof(double2); }

void launch_field_dot(double *out_dev, const void *a, const void *b, Prec p, long n, void *work, cudaStream_t st)
{
    double2 *part = reinterpret_cast<double2 *>(work);
    if (p == P64)
        field_dot_kernel<double><<<kDotCtas, kDotThreads, 0, st>>>((const double *)a, (const double *)b, n, part);
    else
        field_dot_kernel<float><<<kDotCtas, kDotThreads, 0, st>>>((const float *)a, (const float *)b, n, part);
    DWF_CUDA(cudaGetLastError());
    field_dot_reduce<<<1, 32, 0, st>>>(part, reinterpret_cast<double2 *>(out_dev));
    DWF_CUDA(cudaGetLastError());
    count_launch(2);
}

}  // namespace dwf
