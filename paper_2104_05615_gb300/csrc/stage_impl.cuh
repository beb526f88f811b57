// Fused hop stage: one launch applies the Wilson hop D^w (or D^w^+) of
// Sec. 2.2 on one checkerboard, followed by the fifth-dimension matrices that
// follow it in Eq. (eq:detail) of Sec. 3.1.3, and optional axpy terms:
//
//   MODE_F : out = F . hop(in)
//   MODE_S2: out = G . aux - (G F) . hop(in)       (G null: aux - F hop)
//   MODE_S4: out = G . aux - F . hop(in)           (G null: aux - F hop), and a
//            per-CTA partial of <dotv, out> (the <p, Ap> of CG)
//   MODE_5D: out = F . in (no hop)
// with, optionally, M_phi applied to every neighbour as it is loaded.
//
// The four stages of D^+D (Sec. 3.1.3, the five fused kernels) are composed as
//   S1: t1 = [M_phi M5^-1] hop(M_phi x)          (MODE_F, M_phi on load)
//   S2: w  = M5^-+ (x - M5^-1 hop(t1))           (MODE_S2)
//   S3: t3 = [M5^-+ M_phi^+] hop^+(w)            (MODE_F)
//   S4: D^+D x = M5op^+ w - M_phi^+ hop^+(t3)    (MODE_S4; M5op^+ w = D x)
// Each F/G is an Ls x Ls real matrix per chirality.
//
// A CTA owns `tile` output 4D sites and all Ls slices (the Ls-slab of
// Sec. 3.1.3 stays inside one CTA).  Data movement (FP32 / FP16 / BF16):
// threads (j, k) issue bulk asynchronous copies (cp.async.bulk, the TMA
// engine) of the whole Ls-column of neighbour k of site j, the link row of
// site j, the FP16 scales and the aux / dot columns into shared memory,
// completing on one mbarrier; the wait is bounded and raises an error flag
// instead of hanging.  Thread (j, s) then computes the hop of 5D site (j, s)
// from shared memory (the column also holds psi_{s+-1}, so M_phi costs no
// extra loads).  The dense fifth-dimension products run
//   - for FP16/BF16 storage on the tensor cores: [G | -F] (FP16, fixed per
//     system) times [aux ; h] (FP16, scaled by the max-abs of the site as in
//     Sec. 3.1.4) with FP32 accumulation, mma.sync m16n8k16 (Ls padded to 16);
//   - for FP32/FP64 storage on the CUDA cores from shared memory.
// FP64 (used only for reliable updates) loads neighbours directly.
#pragma once

#include <type_traits>

#include "device_common.cuh"

namespace dwf {

constexpr int kLinkStride = 20;  // reals per staged link (18 used, 16-byte aligned)
// reals per site of staged links: its 8 links plus a 16-byte skew, so that the
// links of the (up to three) sites a warp covers fall in different banks
constexpr int kSiteLinkStride = 8 * kLinkStride + 4;
__host__ __device__ constexpr int link_slot(int e) { return (e >> 3) * kSiteLinkStride + (e & 7) * kLinkStride; }

// ------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    uint64_t state;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 %0, [%1], %2;"
                 : "=l"(state)
                 : "r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
    (void)state;
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t phase)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Bounded wait: gives up after `limit` polls (0: 2^22; each poll may suspend
// briefly), records the failure and lets the CTA finish (results are then
// invalid and the host reports DWF_ETIMEOUT).  Returns whether the phase
// completed.
constexpr uint32_t kDefaultPollLimit = 1u << 22;
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t phase, int *err,
                                                  uint32_t limit = 0)
{
    const uint32_t n = limit ? limit : kDefaultPollLimit;
    for (uint32_t it = 0; it < n; it++)
        if (mbar_try_wait(bar, phase)) return true;
    if (err) atomicExch(err, 1);
    return false;
}

// ------------------------------------------------------------- helpers
template <typename R>
__device__ __forceinline__ void load_U(const R *sU, R *u);
template <>
__device__ __forceinline__ void load_U<float>(const float *sU, float *u)
{
    const float4 *p = reinterpret_cast<const float4 *>(sU);
#pragma unroll
    for (int c = 0; c < 4; c++) {
        float4 f = p[c];
        u[4 * c] = f.x;
        u[4 * c + 1] = f.y;
        u[4 * c + 2] = f.z;
        u[4 * c + 3] = f.w;
    }
    float2 f = reinterpret_cast<const float2 *>(sU)[8];
    u[16] = f.x;
    u[17] = f.y;
}
template <>
__device__ __forceinline__ void load_U<double>(const double *sU, double *u)
{
    const double2 *p = reinterpret_cast<const double2 *>(sU);
#pragma unroll
    for (int c = 0; c < 9; c++) {
        double2 f = p[c];
        u[2 * c] = f.x;
        u[2 * c + 1] = f.y;
    }
}

// One direction of the hop on an FP16 colour-spinor in packed half2
// arithmetic: p[spin*3 + colour] = (re, im); U2 holds each link element as
// (re, re), (-im, im).  chi = U h in half2, then accumulated in FP32 with the
// neighbour's weight w (scale times boundary sign).
__device__ __forceinline__ __half2 swap_h2(__half2 z) { return __lowhigh2highlow(z); }
__device__ __forceinline__ uint32_t h2u(__half2 h) { return *reinterpret_cast<uint32_t *>(&h); }
__device__ __forceinline__ __half2 u2h(uint32_t u) { return *reinterpret_cast<__half2 *>(&u); }

template <int MU, int SG>
__device__ __forceinline__ void hop_dir_h2(const __half2 *p, const __half2 *U2, float w, float *acc)
{
    // i z = (-im, re) = swap(z) * (-1, 1)
    const __half2 ipos = __floats2half2_rn(-1.f, 1.f);
    const __half2 ineg = __floats2half2_rn(1.f, -1.f);
    __half2 h[6];  // h[sp*3 + c]
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const __half2 p0 = p[c], p1 = p[3 + c], p2 = p[6 + c], p3 = p[9 + c];
        if constexpr (MU == 0) {  // h0 = p0 + SG i p3, h1 = p1 + SG i p2
            h[c] = __hfma2(swap_h2(p3), SG > 0 ? ipos : ineg, p0);
            h[3 + c] = __hfma2(swap_h2(p2), SG > 0 ? ipos : ineg, p1);
        } else if constexpr (MU == 1) {  // h0 = p0 + SG p3, h1 = p1 - SG p2
            h[c] = SG > 0 ? __hadd2(p0, p3) : __hsub2(p0, p3);
            h[3 + c] = SG > 0 ? __hsub2(p1, p2) : __hadd2(p1, p2);
        } else if constexpr (MU == 2) {  // h0 = p0 + SG i p2, h1 = p1 - SG i p3
            h[c] = __hfma2(swap_h2(p2), SG > 0 ? ipos : ineg, p0);
            h[3 + c] = __hfma2(swap_h2(p3), SG > 0 ? ineg : ipos, p1);
        } else {  // h0 = p0 + SG p2, h1 = p1 + SG p3
            h[c] = SG > 0 ? __hadd2(p0, p2) : __hsub2(p0, p2);
            h[3 + c] = SG > 0 ? __hadd2(p1, p3) : __hsub2(p1, p3);
        }
    }
    __half2 hs[6];
#pragma unroll
    for (int q = 0; q < 6; q++) hs[q] = swap_h2(h[q]);
    float chi[12];  // [sp][row][re, im]
#pragma unroll
    for (int r = 0; r < 3; r++) {
        const __half2 *Ur = U2 + r * 6;
#pragma unroll
        for (int sp = 0; sp < 2; sp++) {
            __half2 t = __hmul2(Ur[0], h[sp * 3]);
            t = __hfma2(Ur[1], hs[sp * 3], t);
            t = __hfma2(Ur[2], h[sp * 3 + 1], t);
            t = __hfma2(Ur[3], hs[sp * 3 + 1], t);
            t = __hfma2(Ur[4], h[sp * 3 + 2], t);
            t = __hfma2(Ur[5], hs[sp * 3 + 2], t);
            const float2 f = __half22float2(t);
            chi[(sp * 3 + r) * 2] = w * f.x;
            chi[(sp * 3 + r) * 2 + 1] = w * f.y;
        }
    }
    accumulate_ct<MU, SG, float>(chi, acc);
}

// The same direction accumulated in half2: acc2[spin*3 + colour] += w2 (chi
// rebuilt to four spins), with w2 the neighbour's weight relative to the
// site's reference scale (|w| <= 1), so the eight directions sum to at most a
// few tens in FP16; the caller converts to FP32 and multiplies by the
// reference once.
template <int MU, int SG>
__device__ __forceinline__ void hop_dir_h2_acc(const __half2 *p, const __half2 *U2, __half2 w2, __half2 *acc2)
{
    const __half2 ipos = __floats2half2_rn(-1.f, 1.f);
    const __half2 ineg = __floats2half2_rn(1.f, -1.f);
    __half2 h[6];  // h[sp*3 + c]
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const __half2 p0 = p[c], p1 = p[3 + c], p2 = p[6 + c], p3 = p[9 + c];
        if constexpr (MU == 0) {  // h0 = p0 + SG i p3, h1 = p1 + SG i p2
            h[c] = __hfma2(swap_h2(p3), SG > 0 ? ipos : ineg, p0);
            h[3 + c] = __hfma2(swap_h2(p2), SG > 0 ? ipos : ineg, p1);
        } else if constexpr (MU == 1) {  // h0 = p0 + SG p3, h1 = p1 - SG p2
            h[c] = SG > 0 ? __hadd2(p0, p3) : __hsub2(p0, p3);
            h[3 + c] = SG > 0 ? __hsub2(p1, p2) : __hadd2(p1, p2);
        } else if constexpr (MU == 2) {  // h0 = p0 + SG i p2, h1 = p1 - SG i p3
            h[c] = __hfma2(swap_h2(p2), SG > 0 ? ipos : ineg, p0);
            h[3 + c] = __hfma2(swap_h2(p3), SG > 0 ? ineg : ipos, p1);
        } else {  // h0 = p0 + SG p2, h1 = p1 + SG p3
            h[c] = SG > 0 ? __hadd2(p0, p2) : __hsub2(p0, p2);
            h[3 + c] = SG > 0 ? __hadd2(p1, p3) : __hsub2(p1, p3);
        }
    }
    __half2 hs[6];
#pragma unroll
    for (int q = 0; q < 6; q++) hs[q] = swap_h2(h[q]);
    // the link's 18 half2 (a 16-byte aligned 80-byte slot) in five wide loads
    __half2 U[18];
    {
        const uint4 *u4 = reinterpret_cast<const uint4 *>(U2);
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const uint4 w = u4[q];
            U[4 * q] = u2h(w.x);
            U[4 * q + 1] = u2h(w.y);
            U[4 * q + 2] = u2h(w.z);
            U[4 * q + 3] = u2h(w.w);
        }
        const uint2 w = reinterpret_cast<const uint2 *>(U2)[8];
        U[16] = u2h(w.x);
        U[17] = u2h(w.y);
    }
    __half2 chi[6];  // [sp][row]
#pragma unroll
    for (int r = 0; r < 3; r++) {
        const __half2 *Ur = U + r * 6;
#pragma unroll
        for (int sp = 0; sp < 2; sp++) {
            __half2 t = __hmul2(Ur[0], h[sp * 3]);
            t = __hfma2(Ur[1], hs[sp * 3], t);
            t = __hfma2(Ur[2], h[sp * 3 + 1], t);
            t = __hfma2(Ur[3], hs[sp * 3 + 1], t);
            t = __hfma2(Ur[4], h[sp * 3 + 2], t);
            t = __hfma2(Ur[5], hs[sp * 3 + 2], t);
            chi[sp * 3 + r] = t;
        }
    }
    // spins 0, 1: + w chi; spins 2, 3 rebuilt (the reconstruction of
    // accumulate_ct): MU=x (-SG i c1, -SG i c0), y (-SG c1, SG c0),
    // z (-SG i c0, SG i c1), t (SG c0, SG c1); -i z = swap(z) (1, -1)
    const __half2 wn = __hneg2(w2);
    const __half2 wmi = __hmul2(w2, ineg);  // w times -i acting on a swapped value
    const __half2 wpi = __hmul2(w2, ipos);  // w times +i acting on a swapped value
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const __half2 c0 = chi[c], c1 = chi[3 + c];
        acc2[c] = __hfma2(w2, c0, acc2[c]);
        acc2[3 + c] = __hfma2(w2, c1, acc2[3 + c]);
        if constexpr (MU == 0) {
            acc2[6 + c] = __hfma2(SG > 0 ? wmi : wpi, swap_h2(c1), acc2[6 + c]);
            acc2[9 + c] = __hfma2(SG > 0 ? wmi : wpi, swap_h2(c0), acc2[9 + c]);
        } else if constexpr (MU == 1) {
            acc2[6 + c] = __hfma2(SG > 0 ? wn : w2, c1, acc2[6 + c]);
            acc2[9 + c] = __hfma2(SG > 0 ? w2 : wn, c0, acc2[9 + c]);
        } else if constexpr (MU == 2) {
            acc2[6 + c] = __hfma2(SG > 0 ? wmi : wpi, swap_h2(c0), acc2[6 + c]);
            acc2[9 + c] = __hfma2(SG > 0 ? wpi : wmi, swap_h2(c1), acc2[9 + c]);
        } else {
            acc2[6 + c] = __hfma2(SG > 0 ? w2 : wn, c0, acc2[6 + c]);
            acc2[9 + c] = __hfma2(SG > 0 ? w2 : wn, c1, acc2[9 + c]);
        }
    }
}

// Decode the NC 16-byte chunks of one 5D spinor (stride `cs` chunks apart);
// kBiased: 16-bit fixed point left as the biased floats of unpack8_fx16_biased.
template <class T, bool kBiased = false>
__device__ __forceinline__ void decode_chunks(const uint4 *p, int cs, typename T::R *v)
{
    if constexpr (T::P == P64) {
#pragma unroll
        for (int c = 0; c < 12; c++) {
            const uint4 w = p[c * cs];
            const double2 d = *reinterpret_cast<const double2 *>(&w);
            v[2 * c] = d.x;
            v[2 * c + 1] = d.y;
        }
    } else if constexpr (T::P == P32) {
#pragma unroll
        for (int c = 0; c < 6; c++) {
            const uint4 w = p[c * cs];
            const float4 f = *reinterpret_cast<const float4 *>(&w);
            v[4 * c] = f.x;
            v[4 * c + 1] = f.y;
            v[4 * c + 2] = f.z;
            v[4 * c + 3] = f.w;
        }
    } else if constexpr (T::P == PFX16) {
#pragma unroll
        for (int c = 0; c < 3; c++) {
            if constexpr (kBiased) unpack8_fx16_biased(p[c * cs], v + 8 * c);
            else unpack8_fx16(p[c * cs], v + 8 * c);
        }
    } else if constexpr (T::P == P16) {
#pragma unroll
        for (int c = 0; c < 3; c++) unpack8(p[c * cs], v + 8 * c, __half());
    } else {
#pragma unroll
        for (int c = 0; c < 3; c++) unpack8(p[c * cs], v + 8 * c, __nv_bfloat16());
    }
}

// acc[r] (+)= coef * sum_t M[chi(r)][s][t] X[t][r] (slice t at X + t * xs);
// MT[t][s] holds (chi0, chi1) pairs
template <typename R, bool kAdd>
__device__ __forceinline__ void apply5(const R *MT, const R *X, int xs, int Ls, int s, R *acc, R coef)
{
    if (!kAdd) {
#pragma unroll
        for (int r = 0; r < 24; r++) acc[r] = 0;
    }
#pragma unroll 2
    for (int t = 0; t < Ls; t++) {
        const R f0 = coef * MT[(t * Ls + s) * 2];
        const R f1 = coef * MT[(t * Ls + s) * 2 + 1];
        const R *x = X + t * xs;
        R xv[24];
        if constexpr (sizeof(R) == 4) {
            const float4 *q = reinterpret_cast<const float4 *>(x);
#pragma unroll
            for (int c = 0; c < 6; c++) {
                float4 f = q[c];
                xv[4 * c] = f.x;
                xv[4 * c + 1] = f.y;
                xv[4 * c + 2] = f.z;
                xv[4 * c + 3] = f.w;
            }
        } else {
            const double2 *q = reinterpret_cast<const double2 *>(x);
#pragma unroll
            for (int c = 0; c < 12; c++) {
                double2 f = q[c];
                xv[2 * c] = f.x;
                xv[2 * c + 1] = f.y;
            }
        }
#pragma unroll
        for (int r = 0; r < 12; r++) acc[r] += f0 * xv[r];
#pragma unroll
        for (int r = 12; r < 24; r++) acc[r] += f1 * xv[r];
    }
}

// Per-(site, s) staging of 24 reals in shared memory (the hop result H and
// the aux column A of the CUDA-core and bidiagonal stages): slice stride an
// odd number of 16-byte units (28 floats, 26 doubles) and a 16-byte skew per
// site, so that neither the slices of one site nor the (up to three) sites of
// a warp share banks.
template <typename R> __host__ __device__ constexpr int slice_stride() { return sizeof(R) == 8 ? 26 : 28; }
template <typename R> __host__ __device__ inline int site_stride(int Ls) { return Ls * slice_stride<R>() + 16 / (int)sizeof(R); }
// Twelve reals from a 16-byte aligned address.
template <typename R>
__device__ __forceinline__ void load12(const R *p, R *v)
{
    if constexpr (sizeof(R) == 4) {
        const float4 *q = reinterpret_cast<const float4 *>(p);
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const float4 f = q[c];
            v[4 * c] = f.x;
            v[4 * c + 1] = f.y;
            v[4 * c + 2] = f.z;
            v[4 * c + 3] = f.w;
        }
    } else {
        const double2 *q = reinterpret_cast<const double2 *>(p);
#pragma unroll
        for (int c = 0; c < 6; c++) {
            const double2 f = q[c];
            v[2 * c] = f.x;
            v[2 * c + 1] = f.y;
        }
    }
}

template <typename R>
__device__ __forceinline__ void store24(R *dst, const R *v)
{
    if constexpr (sizeof(R) == 4) {
        float4 *q = reinterpret_cast<float4 *>(dst);
#pragma unroll
        for (int c = 0; c < 6; c++) q[c] = make_float4(v[4 * c], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3]);
    } else {
#pragma unroll
        for (int r = 0; r < 24; r++) dst[r] = v[r];
    }
}

__device__ __forceinline__ uint32_t pack_h2(float lo, float hi)
{
    __half2 h = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&h);
}

__device__ __forceinline__ void mma_16816(float *d, const uint4 &a, uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a.x), "r"(a.y), "r"(a.z), "r"(a.w), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void mma_1688(float *d, uint32_t a0, uint32_t a1, uint32_t b0)
{
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5}, {%6}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(b0));
}
// Two 8x8 FP16 matrices, transposed: lanes 0..7 address the rows of the
// first, 8..15 of the second (m16n8k8 B fragments of two n-tiles).
__device__ __forceinline__ void ldmatrix_x2_trans(uint32_t addr, uint32_t &r0, uint32_t &r1)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];\n"
                 : "=r"(r0), "=r"(r1)
                 : "r"(addr));
}

// Four 8x8 FP16 matrices from shared memory, transposed: lane l supplies the
// address of row (l & 7) of matrix (l >> 3); register i receives matrix i
// with lane (g, t) holding rows 2t, 2t+1 of column g (an m16n8k16 B fragment).
__device__ __forceinline__ void ldmatrix_x4_trans(uint32_t addr, uint32_t &r0, uint32_t &r1, uint32_t &r2,
                                                  uint32_t &r3)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}

// Fifth-dimension structure (Sec. 2.2): M5op = A + B P with P a one-step
// shift in s, "up" ((P y)_s = y_{s+1}, (P y)_{L-1} = -mass y_0; chirality 0)
// or "down" ((P y)_s = y_{s-1}, (P y)_0 = -mass y_{L-1}; chirality 1); P^T
// swaps the two.  (A + B P)^-1 x: the first element (in the recurrence's
// order) from the closed form of the inverse's first row, then
// y_s = x_s / A + q y_{s-+1}, q = -B/A (|q| < 0.9 is checked on the host, so
// the recurrence damps rounding).  In place on the column x[0..L).
template <typename R, int L>
__device__ __forceinline__ void m5_solve(R *x, bool up, R A, R q, R mass)
{
    const R invA = R(1) / A;
    R qL = R(1);
#pragma unroll
    for (int t = 0; t < L; t++) qL *= q;
    const R invAd = invA / (R(1) + mass * qL);
    R S = R(0);
    if (!up) {
#pragma unroll
        for (int t = 1; t < L; t++) S = q * S + x[t];
        R y = (x[0] - mass * q * S) * invAd;
        x[0] = y;
#pragma unroll
        for (int t = 1; t < L; t++) {
            y = x[t] * invA + q * y;
            x[t] = y;
        }
    } else {
#pragma unroll
        for (int t = L - 2; t >= 0; t--) S = q * S + x[t];
        R y = (x[L - 1] - mass * q * S) * invAd;
        x[L - 1] = y;
#pragma unroll
        for (int t = L - 2; t >= 0; t--) {
            y = x[t] * invA + q * y;
            x[t] = y;
        }
    }
}

// Shared-memory layout of a stage CTA (byte offsets), shared by host and device.
struct StageSmem {
    int bar, nbr, smax, lraw, U, mat, col, scl, aux, auxs, dot, dots, H, A, D, total;
};
__host__ __device__ inline int align16(int x) { return (x + 15) & ~15; }
// Tensor-core operand tiles: FP16 [tile][chi][kt slices][kTcRow(TS) halfs]
// (kt = 16, or 8 for Ls <= 8, whose products use m16n8k8),
// one for h and one for aux; the row pitch is an odd number of 16-byte units
// so the eight rows of an ldmatrix fall in distinct banks.
__host__ __device__ constexpr int kTcRow(int TS) { return TS * 12 + 8; }
// Tensor-core units (chirality x pair of 8-column n-tiles) a warp keeps in
// registers; with more per warp the FP32 output gets its own buffer.
constexpr int kTcMaxUnits = 4;
__host__ __device__ constexpr bool tc_alias(int TS, int Ls)
{
    return (TS * 12 / 8 + (TS * Ls + 31) / 32 - 1) / ((TS * Ls + 31) / 32) <= kTcMaxUnits;
}
__host__ __device__ inline StageSmem stage_smem(int TS, int Ls, int NC, int esz, int rsz, bool tma,
                                                bool tc, bool scale, bool has_aux, bool has_dot,
                                                bool need_ha = true, int kt = 16, bool need_a = true)
{
    // need_ha: the FP32 hop / aux buffers H, A (CUDA-core paths and the
    // bidiagonal S4, which stages one combined buffer: need_a false); the
    // tensor-core stages use the FP16 tiles instead
    StageSmem m;
    const int colb = NC * Ls * 16;
    int o = 0;
    m.bar = o;
    o = align16(o + 8);
    m.nbr = o;
    o = align16(o + TS * 8 * 4);
    m.smax = o;
    o = align16(o + TS * 4);
    m.lraw = o;
    o = align16(o + (tma ? TS * 96 * esz : 0));
    m.U = o;
    o = align16(o + TS * kSiteLinkStride * rsz);
    m.mat = o;
    o = align16(o + (tc ? 0 : 4 * Ls * Ls * rsz));
    m.aux = o;
    o = align16(o + ((tma && has_aux) ? TS * colb : 0));
    m.auxs = o;
    o = align16(o + ((tma && has_aux && scale) ? TS * Ls * 4 : 0));
    m.dot = o;
    o = align16(o + ((tma && has_dot) ? TS * colb : 0));
    m.dots = o;
    o = align16(o + ((tma && has_dot && scale) ? TS * Ls * 4 : 0));
    // neighbour columns; the hop result (H, A or the FP16 tiles) and the
    // tensor-core output alias them afterwards
    const int hb = TS * (Ls * (rsz == 8 ? 26 : 28) + 16 / rsz) * rsz;
    m.col = o;
    m.scl = align16(o + (tma ? TS * 8 * colb : 0));
    int end = align16(m.scl + ((tma && scale) ? TS * 8 * Ls * 4 : 0));
    m.H = o;
    m.A = align16(m.H + hb);
    m.D = o;
    if (need_ha) {
        const int e = align16(m.A + ((has_aux && need_a) ? hb : 0));
        end = e > end ? e : end;
    }
    if (tc) {
        const int bsz = (has_aux ? 2 : 1) * 2 * kt * kTcRow(TS) * 2;
        const int db = TS * Ls * 24 * 2;  // the FP16 result D
        int e;
        if (tc_alias(TS, Ls)) {
            e = align16(o + (bsz > db ? bsz : db));
        } else {
            m.D = align16(o + bsz);
            e = align16(m.D + db);
        }
        end = e > end ? e : end;
    }
    m.total = end;
    return m;
}

// Launch bounds.  The stages are latency-bound on their neighbour gathers,
// so resident warps count for more than the rematerialisation a tight
// register budget costs (measured on GB300).  With precomputed M_phi input:
// FP16 stages of a compile-time shape 56 registers (S4, which keeps more
// values live, 64), the other 16-bit and 8-bit stages 64, FP32 stages of a
// compile-time shape 72.  M_phi on load needs more live values and is not
// bounded, nor is FP64.  With a compile-time launch shape (Ls and tile fixed)
// the block size is exact; shapes fixed only at run time declare 512 threads.
#ifndef DWF_STAGE_REGS_F16
#define DWF_STAGE_REGS_F16 56
#endif
#ifndef DWF_STAGE_REGS_F16_S4
#define DWF_STAGE_REGS_F16_S4 64
#endif
#ifndef DWF_STAGE_REGS_16
#define DWF_STAGE_REGS_16 64
#endif
#ifndef DWF_STAGE_REGS_32
#define DWF_STAGE_REGS_32 72
#endif
template <class T, int kMode, bool kMphi, int LS, int TSC>
struct StageLaunch {
    static constexpr bool kFixed = LS > 0 && TSC > 0;
    static constexpr bool k16 = T::P == P16 || T::P == PB16 || T::P == PFX16 || T::P == PFX8;
    static constexpr int kThreads = kFixed ? (TSC * LS + 31) / 32 * 32 : 512;
    static constexpr int kRegs = kMphi                       ? 0
                                 : (T::P == P16 && kFixed)    ? (kMode == MODE_S4 ? DWF_STAGE_REGS_F16_S4
                                                                                  : DWF_STAGE_REGS_F16)
                                 : k16                        ? DWF_STAGE_REGS_16
                                 : (T::P == P32 && kFixed)    ? DWF_STAGE_REGS_32
                                                              : 0;
    // blocks per SM such that each of the four 16384-register partitions
    // holds its share of the warps at the register budget
    static constexpr int kMinBlocks = kRegs == 0 ? 1
                                      : kFixed ? (16384 / (32 * kRegs)) * 4 / (kThreads / 32)
                                               : 65536 / (512 * kRegs);
};

template <class T, int kMode, bool kMphi, bool kStage, bool kDag, int LS, int TSC>
__global__ void __launch_bounds__(StageLaunch<T, kMode, kMphi, LS, TSC>::kThreads,
                                  StageLaunch<T, kMode, kMphi, LS, TSC>::kMinBlocks)
    stage_kernel(const StageArgs a)
{
    using R = typename T::R;
    constexpr bool kTC = (T::P == P16 || T::P == PB16 || T::P == PFX16 || T::P == PFX8);
    constexpr bool kScale = (T::P == P16 || T::P == PFX16 || T::P == PFX8);
    constexpr bool kTma = kStage && (T::P != P64) && (kMode != MODE_5D);
    // slices per tensor-core operand tile: Ls <= 8 (compile-time) uses 8
    constexpr int KT = (LS > 0 && LS <= 8) ? 8 : 16;
    constexpr bool kAux = (kMode == MODE_S2 || kMode == MODE_S4);
    constexpr int NC = T::NC;
    // FP16 storage (values scaled to [-1, 1] per colour-spinor): projection and
    // SU(3) products in packed half2 arithmetic, accumulation over the eight
    // directions in FP32
    constexpr bool kH2 = (T::P == P16) && !kMphi && !kTma && (kMode != MODE_5D);
    using LE = typename LinkElem<T>::E;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // compile-time fifth extent and tile for the common shapes
    const int Ls = LS > 0 ? LS : a.Ls;
    const int TS = TSC > 0 ? TSC : a.tile;
    const int tid = threadIdx.x;
    const int nthr = (LS > 0 && TSC > 0) ? (TSC * LS + 31) / 32 * 32 : (int)blockDim.x;
    const int jl = tid / Ls;
    const int s = tid - jl * Ls;
    const bool active = jl < TS;
    const long i0 = a.site0 + (long)blockIdx.x * TS;  // absolute: launches may cover a site range
    const long i = i0 + (active ? jl : 0);
    const long cta = i0 / TS;                         // absolute CTA index (dot partials)
    const int sys = a.tile_sys ? a.tile_sys[i0 / kSegPad] : 0;
    if (a.active && !a.active[sys]) {
        // a converged system of a batch: nothing to do (whole CTA, one system)
        if (kMode == MODE_S4 && a.dot_part && tid == 0) a.dot_part[cta] = 0.0;
        return;
    }
    const bool has_dot = (kMode == MODE_S4) && a.dot_part;
    const bool scale_bulk = kScale && (Ls % 4 == 0);
    const StageSmem L = stage_smem(TS, Ls, NC, sizeof(LE), sizeof(R), kTma, kTC, scale_bulk, kAux,
                                   has_dot, !kTC || kMode == MODE_S4, KT, kMode != MODE_S4);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem_raw + L.bar);
    int *sN = reinterpret_cast<int *>(smem_raw + L.nbr);
    float *sMax = reinterpret_cast<float *>(smem_raw + L.smax);
    R *sU = reinterpret_cast<R *>(smem_raw + L.U);
    R *sX = reinterpret_cast<R *>(smem_raw + L.mat);
    R *sH = reinterpret_cast<R *>(smem_raw + L.H);
    R *sA = reinterpret_cast<R *>(smem_raw + L.A);
    const int hsl = slice_stride<R>(), hsite = site_stride<R>(Ls);
    auto hofs = [&](int j, int t) { return j * hsite + t * hsl; };
    const int colb = NC * Ls * 16;
    const uint4 *sCol = reinterpret_cast<const uint4 *>(smem_raw + L.col);
    const float *sScl = reinterpret_cast<const float *>(smem_raw + L.scl);

    // segments are whole multiples of kSegPad sites and TS divides kSegPad:
    // a CTA never straddles two segments
    const int seg = (int)i0 / a.seg_out;
    const int loc = (int)i - seg * a.seg_out;

    // fifth-dimension matrices for the CUDA-core path, transposed to [t][s][chi]
    auto stage_mats = [&]() {
        const R *Fg = reinterpret_cast<const R *>(a.F) + (size_t)sys * 2 * Ls * Ls;
        const R *Gg = a.G ? reinterpret_cast<const R *>(a.G) + (size_t)sys * 2 * Ls * Ls : nullptr;
        for (int e = tid; e < 2 * Ls * Ls; e += nthr) {
            const int chi = e / (Ls * Ls), rem = e - chi * Ls * Ls;
            const int ss = rem / Ls, t = rem - ss * Ls;
            sX[(t * Ls + ss) * 2 + chi] = Fg[e];
            if (Gg) sX[2 * Ls * Ls + (t * Ls + ss) * 2 + chi] = Gg[e];
        }
    };

    // ---- 1. gather (bulk copies for FP32/16-bit, direct loads for FP64)
    if constexpr (kTma) {
        if (tid == 0) {
            mbar_init(bar, TS * 8);
            fence_mbar_init();
        }
        if (kTC && tid < TS) sMax[tid] = 0.f;
        __syncthreads();
        for (int e = tid; e < TS * 8; e += nthr) {
            const int j = e >> 3, k = e & 7;
            const int ii = (int)i0 + j;
            const int sg_ = seg, lc = ii - sg_ * a.seg_out;
            const int nb = __ldg(a.nbr + (long)ii * 8 + k);
            sN[e] = nb;
            uint32_t bytes = 0;
            const bool link = (k == 0);
            const bool col = nb != -1;
            const long idx = nb >= 0 ? (long)nb : (long)(-nb - 2);
            // own aux / dot columns, issued by k = 1 / k = 2
            const long ai = (long)sg_ * a.aux_stride + lc;
            const bool aux = kAux && k == 1 && (kMode == MODE_S4 || lc < a.aux_valid);
            const bool dot = (kMode == MODE_S4) && k == 2 && a.dot_part;
            const uint32_t sb = scale_bulk ? Ls * 4 : 0;
            if (link) bytes += 96 * sizeof(LE);
            if (col) bytes += colb + sb;
            if (aux) bytes += colb + sb;
            if (dot) bytes += colb + sb;
            mbar_arrive_expect_tx(bar, bytes);
            if (link) {
                const long row = (long)sg_ * a.link_stride + lc;
                bulk_g2s(smem_raw + L.lraw + j * 96 * sizeof(LE),
                         reinterpret_cast<const LE *>(a.links) + row * 96, 96 * sizeof(LE), bar);
            }
            if (col) {
                bulk_g2s(smem_raw + L.col + e * colb, reinterpret_cast<const char *>(a.in) + idx * colb,
                         colb, bar);
                if (scale_bulk)
                    bulk_g2s(smem_raw + L.scl + e * Ls * 4, scale_ptr<TF16>(a.in, a.nin, Ls) + idx * Ls,
                             sb, bar);
            }
            if (aux) {
                bulk_g2s(smem_raw + L.aux + j * colb, reinterpret_cast<const char *>(a.aux) + ai * colb,
                         colb, bar);
                if (scale_bulk)
                    bulk_g2s(smem_raw + L.auxs + j * Ls * 4, scale_ptr<TF16>(a.aux, a.naux, Ls) + ai * Ls,
                             sb, bar);
            }
            if (dot) {
                bulk_g2s(smem_raw + L.dot + j * colb, reinterpret_cast<const char *>(a.dotv) + ii * colb,
                         colb, bar);
                if (scale_bulk)
                    bulk_g2s(smem_raw + L.dots + j * Ls * 4, scale_ptr<TF16>(a.dotv, a.nout, Ls) + ii * Ls,
                             sb, bar);
            }
        }
        if (!kTC) stage_mats();
        mbar_wait_bounded(bar, 0, a.err, a.poll_limit);
        // testing the failure path: every copy has landed (phase 0 is
        // complete); phase 1 is never armed, so this wait runs out
        if (a.force_timeout) mbar_wait_bounded(bar, 1, a.err, a.poll_limit);
        // rebuild the third row of each staged link
        for (int e = tid; e < TS * 8; e += nthr) {
            const int j = e >> 3, k = e & 7;
            R u[18];
            const LE *lr = reinterpret_cast<const LE *>(smem_raw + L.lraw) + j * 96 + k * 12;
#pragma unroll
            for (int q = 0; q < 12; q++) {
                if constexpr (sizeof(LE) == 2) u[q] = (R)__half2float(*reinterpret_cast<const __half *>(lr + q));
                else u[q] = (R)lr[q];
            }
            reconstruct_row2<R>(u);
            R *dst = sU + link_slot(e);
#pragma unroll
            for (int q = 0; q < 18; q++) dst[q] = u[q];
        }
        __syncthreads();
    } else {
        if (kMode != MODE_5D) {
            for (int e = tid; e < TS * 8; e += nthr) {
                const int j = e >> 3, k = e & 7;
                const int ii = (int)i0 + j;
                const long row = (long)seg * a.link_stride + (ii - seg * a.seg_out);
                const int nb = __ldg(a.nbr + (long)ii * 8 + k);
                sN[e] = nb;
                R u[18];
                if (nb != -1) {
                    load_link12<T>(a.links, row, k, u);
                    reconstruct_row2<R>(u);
                } else {
#pragma unroll
                    for (int q = 0; q < 18; q++) u[q] = 0;
                }
                if constexpr (kH2) {
                    // each element as two half2: (re, re) and (-im, im)
                    __half2 *dst = reinterpret_cast<__half2 *>(sU + link_slot(e));
#pragma unroll
                    for (int q = 0; q < 9; q++) {
                        dst[2 * q] = __floats2half2_rn(u[2 * q], u[2 * q]);
                        dst[2 * q + 1] = __floats2half2_rn(-u[2 * q + 1], u[2 * q + 1]);
                    }
                } else {
                    R *dst = sU + link_slot(e);
#pragma unroll
                    for (int q = 0; q < 18; q++) dst[q] = u[q];
                }
            }
        }
        if (kTC && tid < TS) sMax[tid] = 0.f;
        if (!kTC) stage_mats();
        __syncthreads();
    }

    // ---- 2. hop
    R acc[24];
#pragma unroll
    for (int r = 0; r < 24; r++) acc[r] = 0;
    if (kMode == MODE_5D) {
        if (active) load_sp<T>(a.in, a.nin, i, s, Ls, acc);
    } else if (active) {
        R cb = 0, cc = 0, wm = 0;
        if (kMphi) {
            const double *mp = a.mphi + 5 * sys;
            cb = (R)(-0.5 * mp[0]);
            cc = (R)(-0.5 * mp[1]);
            wm = (R)(-mp[2]);
        }
        const int sp = s + 1 < Ls ? s + 1 : 0;
        const int sm1 = s > 0 ? s - 1 : Ls - 1;
        // the site's eight neighbour entries in two 16-byte shared loads
        int nb8[8];
        {
            const int4 *q = reinterpret_cast<const int4 *>(sN + jl * 8);
            const int4 x0 = q[0], x1 = q[1];
            nb8[0] = x0.x; nb8[1] = x0.y; nb8[2] = x0.z; nb8[3] = x0.w;
            nb8[4] = x1.x; nb8[5] = x1.y; nb8[6] = x1.z; nb8[7] = x1.w;
        }
        // FP16 path: the eight directions accumulate in half2 relative to the
        // largest neighbour scale at this (site, s)
        float scl[8];
        float inv_ref = 0.f, ref = 0.f;
        __half2 acc2[12];
        if constexpr (kH2) {
#pragma unroll
            for (int k = 0; k < 8; k++) {
                const int e = nb8[k];
                scl[k] = 0.f;
                if (e != -1) {
                    const long idx = e >= 0 ? (long)e : (long)(-e - 2);
                    scl[k] = __ldg(scale_ptr<TF16>(a.in, a.nin, Ls) + idx * Ls + s);
                    ref = fmaxf(ref, scl[k]);
                }
            }
            inv_ref = ref > 0.f ? __fdividef(1.f, ref) : 0.f;
#pragma unroll
            for (int q = 0; q < 12; q++) acc2[q] = __float2half2_rn(0.f);
        }
        // one direction k = 2 mu + d with compile-time mu and projector sign:
        // forward (d = 0) 1 - gamma, backward 1 + gamma, flipped for D^w^+
        auto dir = [&](auto kc) {
            constexpr int k = decltype(kc)::value;
            constexpr int mu = k >> 1;
            constexpr int SG = ((k & 1) ? 1 : -1) * (kDag ? -1 : 1);
            // fixed point: the projection takes the offset of the biased
            // integers off itself (exactly), except where M_phi mixes slices
            constexpr bool kFxB = (T::P == PFX16) && !kMphi;
            const int e = nb8[k];
            if (e == -1) return;
            const long idx = e >= 0 ? (long)e : (long)(-e - 2);
            R psi[24];
            R sc = 1;
            if constexpr (kTma) {
                const uint4 *cp = sCol + (size_t)(jl * 8 + k) * (colb / 16);
                decode_chunks<T, kFxB>(cp + s, Ls, psi);
                if (kScale) {
                    sc = scale_bulk ? sScl[(jl * 8 + k) * Ls + s]
                                    : __ldg(scale_ptr<TF16>(a.in, a.nin, Ls) + idx * Ls + s);
                }
                if (kMphi) {
                    // (M_phi psi)_s = -(b psi_s + c (P_- psi_{s+1} + P_+ psi_{s-1}))/2,
                    // wrap terms times -mass; P_- = spins 0,1, P_+ = spins 2,3
                    R q[24];
                    R s1 = 1, s2 = 1;
                    if (kScale) {
                        s1 = scale_bulk ? sScl[(jl * 8 + k) * Ls + sp]
                                        : __ldg(scale_ptr<TF16>(a.in, a.nin, Ls) + idx * Ls + sp);
                        s2 = scale_bulk ? sScl[(jl * 8 + k) * Ls + sm1]
                                        : __ldg(scale_ptr<TF16>(a.in, a.nin, Ls) + idx * Ls + sm1);
                    }
                    const R fp = (s + 1 < Ls ? cc : cc * wm) * s1;
                    const R fm = (s > 0 ? cc : cc * wm) * s2;
                    const R c0 = cb * sc;
                    decode_chunks<T>(cp + sp, Ls, q);
#pragma unroll
                    for (int r = 0; r < 12; r++) psi[r] = c0 * psi[r] + fp * q[r];
                    decode_chunks<T>(cp + sm1, Ls, q);
#pragma unroll
                    for (int r = 12; r < 24; r++) psi[r] = c0 * psi[r] + fm * q[r];
                    sc = 1;
                }
            } else if constexpr (kH2) {
                const uint4 *gp = reinterpret_cast<const uint4 *>(a.in) + (size_t)idx * NC * Ls;
                uint4 raw[NC];
#pragma unroll
                for (int c = 0; c < NC; c++) raw[c] = __ldg(gp + (size_t)c * Ls + s);
                const float w = (e >= 0 ? scl[k] : -scl[k]) * inv_ref;
                hop_dir_h2_acc<mu, SG>(reinterpret_cast<const __half2 *>(raw),
                                       reinterpret_cast<const __half2 *>(sU + link_slot(jl * 8 + k)),
                                       __float2half2_rn(w), acc2);
                return;
            } else if constexpr (T::P == PFX8) {
                // 8-bit fixed point: three 8-byte chunks per 5D site
                const uint2 *gp = reinterpret_cast<const uint2 *>(a.in) + (size_t)idx * 3 * Ls;
                const float *gs = scale_ptr<TFX8>(a.in, a.nin, Ls) + idx * Ls;
                auto ld = [&](int ss, float *v) {
#pragma unroll
                    for (int c = 0; c < 3; c++) unpack8_fx8(__ldg(gp + (size_t)c * Ls + ss), v + 8 * c);
                    return __ldg(gs + ss);
                };
                sc = ld(s, psi);
                if (kMphi) {
                    R q[24];
                    const R c0 = cb * sc;
                    const R fp = (s + 1 < Ls ? cc : cc * wm) * ld(sp, q);
#pragma unroll
                    for (int r = 0; r < 12; r++) psi[r] = c0 * psi[r] + fp * q[r];
                    const R fm = (s > 0 ? cc : cc * wm) * ld(sm1, q);
#pragma unroll
                    for (int r = 12; r < 24; r++) psi[r] = c0 * psi[r] + fm * q[r];
                    sc = 1;
                }
            } else {
                const uint4 *gp = reinterpret_cast<const uint4 *>(a.in) + (size_t)idx * NC * Ls;
                uint4 raw[NC];
#pragma unroll
                for (int c = 0; c < NC; c++) raw[c] = __ldg(gp + (size_t)c * Ls + s);
                if (kScale) sc = __ldg(scale_ptr<TF16>(a.in, a.nin, Ls) + idx * Ls + s);
                decode_chunks<T, kFxB>(raw, 1, psi);
                if (kMphi) {
                    R q[24];
                    R s1 = 1, s2 = 1;
                    if (kScale) {
                        s1 = __ldg(scale_ptr<TF16>(a.in, a.nin, Ls) + idx * Ls + sp);
                        s2 = __ldg(scale_ptr<TF16>(a.in, a.nin, Ls) + idx * Ls + sm1);
                    }
                    const R fp = (s + 1 < Ls ? cc : cc * wm) * s1;
                    const R fm = (s > 0 ? cc : cc * wm) * s2;
                    const R c0 = cb * sc;
#pragma unroll
                    for (int c = 0; c < NC; c++) raw[c] = __ldg(gp + (size_t)c * Ls + sp);
                    decode_chunks<T>(raw, 1, q);
#pragma unroll
                    for (int r = 0; r < 12; r++) psi[r] = c0 * psi[r] + fp * q[r];
#pragma unroll
                    for (int c = 0; c < NC; c++) raw[c] = __ldg(gp + (size_t)c * Ls + sm1);
                    decode_chunks<T>(raw, 1, q);
#pragma unroll
                    for (int r = 12; r < 24; r++) psi[r] = c0 * psi[r] + fm * q[r];
                    sc = 1;
                }
            }
            R h[12], chi[12];
            project_ct<mu, SG, R, kFxB>(psi, e >= 0 ? sc : -sc, h);
            su3_mul_half_smem<R>(sU + link_slot(jl * 8 + k), h, chi);
            accumulate_ct<mu, SG, R>(chi, acc);
        };
        dir(std::integral_constant<int, 0>{});
        dir(std::integral_constant<int, 1>{});
        dir(std::integral_constant<int, 2>{});
        dir(std::integral_constant<int, 3>{});
        dir(std::integral_constant<int, 4>{});
        dir(std::integral_constant<int, 5>{});
        dir(std::integral_constant<int, 6>{});
        dir(std::integral_constant<int, 7>{});
        if constexpr (kH2) {
#pragma unroll
            for (int q = 0; q < 12; q++) {
                const float2 f = __half22float2(acc2[q]);
                acc[2 * q] = f.x * ref;
                acc[2 * q + 1] = f.y * ref;
            }
        }
    }

    // own aux column; the S2 tensor-core stage on FP16 storage keeps it as
    // stored (normalised half values and their scale, which is also their
    // max-abs) and feeds it to the operand tile in half2 arithmetic
    constexpr bool kAuxRaw = (T::P == P16) && !kTma && kMode == MODE_S2;
    R av[24];
#pragma unroll
    for (int r = 0; r < 24; r++) av[r] = 0;
    uint4 araw[3] = {make_uint4(0u, 0u, 0u, 0u), make_uint4(0u, 0u, 0u, 0u), make_uint4(0u, 0u, 0u, 0u)};
    float asc = 0.f;
    if (kAux) {
        const bool aux_here = (kMode == MODE_S4) || loc < a.aux_valid;
        if (active && aux_here) {
            if constexpr (kAuxRaw) {
                const long ai = (long)seg * a.aux_stride + loc;
                const uint4 *ap = reinterpret_cast<const uint4 *>(a.aux) + (size_t)ai * 3 * Ls + s;
#pragma unroll
                for (int c = 0; c < 3; c++) araw[c] = __ldg(ap + (size_t)c * Ls);
                asc = __ldg(scale_ptr<TF16>(a.aux, a.naux, Ls) + (size_t)ai * Ls + s);
            } else if constexpr (kTma) {
                decode_chunks<T>(reinterpret_cast<const uint4 *>(smem_raw + L.aux) + jl * (colb / 16) + s, Ls, av);
                if (kScale) {
                    const float sa = scale_bulk ? reinterpret_cast<const float *>(smem_raw + L.auxs)[jl * Ls + s]
                                                : __ldg(scale_ptr<TF16>(a.aux, a.naux, Ls) +
                                                        (seg * a.aux_stride + loc) * Ls + s);
#pragma unroll
                    for (int r = 0; r < 24; r++) av[r] *= sa;
                }
            } else {
                load_sp<T>(a.aux, a.naux, seg * a.aux_stride + loc, s, Ls, av);
            }
        }
    }
    if (kTma) {
        // the neighbour columns (written by the async proxy) are reused below
        fence_proxy_async_smem();
        __syncthreads();
    }

    R out[24];
    if constexpr (kMode == MODE_S4) {
        // ---------------------------------------------------------------
        // S4: out = M5op^+ aux - M_phi^+ h with both matrices bidiagonal per
        // chirality: out = A aux + B P^T aux + (b h + c P^T h) / 2, where
        // (P^T v)_s = v_{s-1} on spins 0,1 and v_{s+1} on spins 2,3 (wrap
        // terms times -mass).  G null (the D^+ operator): out = aux + (b h + c P^T h)/2.
        // The shifted terms share one factor per slice (1, or -mass on the
        // wrap), so each (site, s) stages q = B aux + (c/2) h once and reads
        // the neighbouring slices' halves of q.
        const double *mp = a.mphi + 5 * sys;
        const R hb = (R)(0.5 * mp[0]), hc = (R)(0.5 * mp[1]), mass = (R)mp[2];
        const R cA = a.G ? (R)mp[3] : R(1), cB = a.G ? (R)mp[4] : R(0);
        if (active) {
            R q[24];
#pragma unroll
            for (int r = 0; r < 24; r++) q[r] = cB * av[r] + hc * acc[r];
            store24(sH + hofs(jl, s), q);
        }
        __syncthreads();
        if (active) {
            const int sm = s > 0 ? s - 1 : Ls - 1, sp = s + 1 < Ls ? s + 1 : 0;
            const R flo = s > 0 ? R(1) : -mass, fhi = s + 1 < Ls ? R(1) : -mass;
            // the thread's own slice from registers, the neighbouring slices'
            // halves from shared memory
            R Qm[12], Qp[12];
            load12(sH + hofs(jl, sm), Qm);
            load12(sH + hofs(jl, sp) + 12, Qp);
#pragma unroll
            for (int r = 0; r < 12; r++) out[r] = cA * av[r] + hb * acc[r] + flo * Qm[r];
#pragma unroll
            for (int r = 12; r < 24; r++) out[r] = cA * av[r] + hb * acc[r] + fhi * Qp[r - 12];
        }
    } else if constexpr (kTC) {
        // ---------------------------------------------------------------
        // tensor-core path, per chirality D = A . B with A = [G | -F] (FP16
        // fragments fixed per system; M = output slice, K = input slice) and
        // B = [aux ; h] (K = slice, N = site x 12 components).  Each site's hop
        // result and aux column are scaled by their max-abs (Sec. 3.1.4),
        // written once as FP16 rows of the B tiles and read back as fragments
        // with ldmatrix.trans; D is rescaled by the same factor.
        const int RS = kTcRow(TS);
        constexpr int nk = kAux ? 2 : 1;
        // S2 reads aux only on the block interior, which comes first in E2: a
        // tile whose first site lies beyond it has no aux and skips that k-step
        const bool aux_tile = kAux && (kMode == MODE_S4 || (int)(i0 - (long)seg * a.seg_out) < a.aux_valid);
        __half *sB = reinterpret_cast<__half *>(smem_raw + L.H);
        {
            float m = 0.f;
            if (active) {
#pragma unroll
                for (int r = 0; r < 24; r++) m = fmaxf(m, fabsf(acc[r]));
                if constexpr (kAuxRaw) {
                    m = fmaxf(m, asc);
                } else if constexpr (kAux) {
#pragma unroll
                    for (int r = 0; r < 24; r++) m = fmaxf(m, fabsf(av[r]));
                }
            }
            // the lanes of one site are consecutive (at most 16 of them in a
            // warp): a segmented maximum by shuffles leaves the site's maximum
            // in its first lane, which alone updates the shared value (one
            // atomic per site and warp instead of one per thread)
            const int lane = tid & 31;
#pragma unroll
            for (int off = 1; off < 16; off <<= 1) {
                const float o = __shfl_down_sync(0xffffffffu, m, off);
                const int oj = __shfl_down_sync(0xffffffffu, jl, off);
                if (lane + off < 32 && oj == jl) m = fmaxf(m, o);
            }
            const int jprev = __shfl_up_sync(0xffffffffu, jl, 1);
            if (active && (lane == 0 || jprev != jl))
                atomicMax(reinterpret_cast<int *>(sMax + jl), __float_as_int(m));
        }
        {
            // slices Ls..15 of every tile are zero (K padded to 16)
            const int padq = (KT - Ls) * RS / 8;
            for (int e = tid; e < nk * 2 * padq; e += nthr) {
                const int tl = e / padq, q = e - tl * padq;
                reinterpret_cast<uint4 *>(sB + ((size_t)tl * KT + Ls) * RS)[q] = make_uint4(0u, 0u, 0u, 0u);
            }
        }
        __syncthreads();
        if (active) {
            const float sig = sMax[jl];
            // any factor within a few ulp of 1/sig keeps the FP16 operands in range
            const float inv = sig > 0.f ? __fdividef(1.f, sig) : 0.f;
            auto put = [&](__half *tile, const R *v) {
#pragma unroll
                for (int chi = 0; chi < 2; chi++) {
                    uint2 *dst = reinterpret_cast<uint2 *>(tile + ((size_t)chi * KT + s) * RS + jl * 12);
#pragma unroll
                    for (int q = 0; q < 3; q++) {
                        const R *w = v + chi * 12 + 4 * q;
                        dst[q] = make_uint2(pack_h2(w[0] * inv, w[1] * inv), pack_h2(w[2] * inv, w[3] * inv));
                    }
                }
            };
            // tile 0: aux (if any) else h ; tile 1: h
            if (kAux && !aux_tile) {
                put(sB + (size_t)2 * KT * RS, acc);
            } else if constexpr (kAuxRaw) {
                // stored halves times (aux scale / site scale) <= 1
                const __half2 r2 = __float2half2_rn(asc * inv);
                auto mul = [&](uint32_t w) {
                    __half2 h = *reinterpret_cast<const __half2 *>(&w);
                    h = __hmul2(h, r2);
                    return *reinterpret_cast<uint32_t *>(&h);
                };
                // chirality 0 = halves 0..11, chirality 1 = halves 12..23
                uint2 *d0 = reinterpret_cast<uint2 *>(sB + (size_t)s * RS + jl * 12);
                uint2 *d1 = reinterpret_cast<uint2 *>(sB + ((size_t)KT + s) * RS + jl * 12);
                d0[0] = make_uint2(mul(araw[0].x), mul(araw[0].y));
                d0[1] = make_uint2(mul(araw[0].z), mul(araw[0].w));
                d0[2] = make_uint2(mul(araw[1].x), mul(araw[1].y));
                d1[0] = make_uint2(mul(araw[1].z), mul(araw[1].w));
                d1[1] = make_uint2(mul(araw[2].x), mul(araw[2].y));
                d1[2] = make_uint2(mul(araw[2].z), mul(araw[2].w));
                put(sB + (size_t)2 * KT * RS, acc);
            } else if (kAux) {
                put(sB, av);
                put(sB + (size_t)2 * KT * RS, acc);
            } else {
                put(sB, acc);
            }
        }
        __syncthreads();
        const int lane = tid & 31, warp = tid >> 5, nwarp = nthr >> 5;
        const int g = lane >> 2, tg = lane & 3;
        const int npair = TS * 12 / 16;  // pairs of 8-column n-tiles per chirality
        const int nunit = 2 * npair;
        const uint4 *Af = reinterpret_cast<const uint4 *>(a.F) + (size_t)sys * 2 * 2 * 32;
        // this lane's ldmatrix row: slice lr of n-tile ln / 8 of the pair
        const int lr = (lane & 7) + 8 * ((lane >> 3) & 1);
        const int ln = 8 * (lane >> 4);
        const bool alias = tc_alias(TS, Ls);
        R *sD = reinterpret_cast<R *>(smem_raw + L.D);
        auto unit_mma = [&](int u, float *d) {
            const int chi = u / npair, pr = u - chi * npair;
#pragma unroll
            for (int q = 0; q < 8; q++) d[q] = 0.f;
#pragma unroll
            for (int kk = 0; kk < nk; kk++) {
                if (kAux && kk == 0 && !aux_tile) continue;  // aux all zero in this tile
                // A fragment of this lane, [G | -F] of this chirality and k-step
                const uint4 af = __ldg(Af + ((chi * 2 + kk) * 32 + lane));
                if constexpr (KT == 8) {
                    // K = 8 slices: the first two registers of the k16 fragment
                    // are the m16n8k8 A fragment (columns 0..7)
                    const __half *tb = sB + ((size_t)(kk * 2 + chi) * 8 + (lane & 7)) * RS + pr * 16 +
                                       8 * ((lane >> 3) & 1);
                    uint32_t b0, b1;
                    ldmatrix_x2_trans(smem_u32(tb), b0, b1);
                    mma_1688(d, af.x, af.y, b0);
                    mma_1688(d + 4, af.x, af.y, b1);
                } else {
                    const __half *tb = sB + ((size_t)(kk * 2 + chi) * 16 + lr) * RS + pr * 16 + ln;
                    uint32_t b0, b1, b2, b3;
                    ldmatrix_x4_trans(smem_u32(tb), b0, b1, b2, b3);
                    mma_16816(d, af, b0, b1);
                    mma_16816(d + 4, af, b2, b3);
                }
            }
        };
        auto unit_store = [&](int u, const float *d) {
            // D rows s = g, g + 8 ; columns 2 tg, 2 tg + 1 of each n-tile -> one site
            const int chi = u / npair, pr = u - chi * npair;
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const int nd = pr * 16 + h * 8 + 2 * tg;
                const int jd = nd / 12, rd = chi * 12 + (nd - jd * 12);
                // D is normalised by the site scale (the scaled formats fold
                // that scale into the stored one, BF16 multiplies it back when
                // reading D), so it is kept as FP16
                __half *sDh = reinterpret_cast<__half *>(sD);
                if (g < Ls)
                    *reinterpret_cast<uint32_t *>(sDh + (jd * Ls + g) * 24 + rd) = pack_h2(d[4 * h], d[4 * h + 1]);
                if (g + 8 < Ls)
                    *reinterpret_cast<uint32_t *>(sDh + (jd * Ls + g + 8) * 24 + rd) =
                        pack_h2(d[4 * h + 2], d[4 * h + 3]);
            }
        };
        if (alias) {
            // the units of this warp stay in registers while the output
            // overwrites the operand tiles
            float dreg[kTcMaxUnits][8];
#pragma unroll
            for (int u = 0; u < kTcMaxUnits; u++) {
                const int uu = warp + u * nwarp;
                if (uu < nunit) unit_mma(uu, dreg[u]);
            }
            __syncthreads();  // every warp has read the tiles
#pragma unroll
            for (int u = 0; u < kTcMaxUnits; u++) {
                const int uu = warp + u * nwarp;
                if (uu < nunit) unit_store(uu, dreg[u]);
            }
        } else {
            for (int uu = warp; uu < nunit; uu += nwarp) {
                float d[8];
                unit_mma(uu, d);
                unit_store(uu, d);
            }
        }
        __syncthreads();
        if (active) {
            const uint4 *q4 = reinterpret_cast<const uint4 *>(reinterpret_cast<const __half *>(sD) +
                                                              (jl * Ls + s) * 24);
#pragma unroll
            for (int c = 0; c < 3; c++) unpack8(q4[c], out + 8 * c, __half());
            if constexpr (!kScale) {
                const float sd = sMax[jl];
#pragma unroll
                for (int r = 0; r < 24; r++) out[r] *= sd;
            }
        }
    } else {
        // ---------------------------------------------------------------
        // CUDA-core path (FP32 / FP64)
        const R *sF = sX, *sG = sX + 2 * Ls * Ls;
        // (the structured programs read the per-system b, c, mass, A, B)
        const bool structured = LS > 0 && a.fprog != FP_DENSE && a.mphi != nullptr;
        if (active) {
            store24(sH + hofs(jl, s), acc);
            if (kAux && (a.G || structured)) store24(sA + hofs(jl, s), av);
        }
        __syncthreads();
        if constexpr (LS > 0) {
            if (structured) {
                // one thread per (site, real component) runs the column's
                // fifth-dimension program in place, then every (site, s)
                // thread reads its 24 outputs back
                const double *mp = a.mphi + 5 * sys;
                const R mass = (R)mp[2], A5 = (R)mp[3], q = (R)(-mp[4] / mp[3]);
                for (int col = tid; col < TS * 24; col += nthr) {
                    const int j = col / 24, r = col - j * 24;
                    const bool up = r < 12;  // chirality 0: spins 0, 1
                    R x[LS];
#pragma unroll
                    for (int t = 0; t < LS; t++) x[t] = sH[hofs(j, t) + r];
                    switch (a.fprog) {
                    case FP_M5I: m5_solve<R, LS>(x, up, A5, q, mass); break;
                    case FP_M5ID: m5_solve<R, LS>(x, !up, A5, q, mass); break;
                    default:  // FP_S2
                        m5_solve<R, LS>(x, up, A5, q, mass);
#pragma unroll
                        for (int t = 0; t < LS; t++) x[t] = sA[hofs(j, t) + r] - x[t];
                        m5_solve<R, LS>(x, !up, A5, q, mass);
                        break;
                    }
                    if (kMode == MODE_S2 && a.fprog != FP_S2) {
                        // G null: aux - F h
#pragma unroll
                        for (int t = 0; t < LS; t++) x[t] = sA[hofs(j, t) + r] - x[t];
                    }
#pragma unroll
                    for (int t = 0; t < LS; t++) sH[hofs(j, t) + r] = x[t];
                }
                __syncthreads();
                if (active) {
#pragma unroll
                    for (int r = 0; r < 24; r++) out[r] = sH[hofs(jl, s) + r];
                }
            }
        }
        const R *Hsite = sH + hofs(jl, 0);
        if (active && !structured) {
            if (kMode == MODE_F || kMode == MODE_5D) {
                apply5<R, false>(sF, Hsite, hsl, Ls, s, out, R(1));
            } else {
                // MODE_S2: out = G aux - F' h  (F' = G F; G null: aux - F h)
                if (a.G) {
                    apply5<R, false>(sG, sA + hofs(jl, 0), hsl, Ls, s, out, R(1));
                } else {
#pragma unroll
                    for (int r = 0; r < 24; r++) out[r] = av[r];
                }
                apply5<R, true>(sF, Hsite, hsl, Ls, s, out, R(-1));
            }
        }
    }

    if constexpr (kTC && kScale && kMode != MODE_S4) {
        // out holds D / (site scale): the factor goes into the stored scale
        if (active) store_sp_scaled<T>(a.out, a.nout, i, s, Ls, out, sMax[jl]);
    } else {
        if (active) store_sp<T>(a.out, a.nout, i, s, Ls, out);
    }

    if (kMode == MODE_S4 && a.dot_part) {
        // partial <dotv, out> (real part), per thread in R, across threads in FP64
        R dsum = 0;
        if (active) {
            R pv[24];
            if constexpr (kTma) {
                decode_chunks<T>(reinterpret_cast<const uint4 *>(smem_raw + L.dot) + jl * (colb / 16) + s, Ls, pv);
                if (kScale) {
                    const float sd = scale_bulk ? reinterpret_cast<const float *>(smem_raw + L.dots)[jl * Ls + s]
                                                : __ldg(scale_ptr<TF16>(a.dotv, a.nout, Ls) + i * Ls + s);
#pragma unroll
                    for (int r = 0; r < 24; r++) pv[r] *= sd;
                }
            } else {
                load_sp<T>(a.dotv, a.nout, i, s, Ls, pv);
            }
#pragma unroll
            for (int r = 0; r < 24; r++) dsum += pv[r] * out[r];
        }
        double dd = (double)dsum;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) dd += __shfl_xor_sync(0xffffffffu, dd, o);
        __shared__ double red[32];
        if ((tid & 31) == 0) red[tid >> 5] = dd;
        __syncthreads();
        if (tid < 32) {
            double v = tid < (nthr + 31) / 32 ? red[tid] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (tid == 0) a.dot_part[cta] = v;
        }
    }
}

template <class T, int kMode, bool kMphi, bool kStage, bool kDag, int LS, int TSC>
static void launch_t(const StageArgs &a, cudaStream_t st)
{
    using R = typename T::R;
    using LE = typename LinkElem<T>::E;
    constexpr bool kTC = (T::P == P16 || T::P == PB16 || T::P == PFX16 || T::P == PFX8);
    constexpr bool kTma = kStage && (T::P != P64) && (kMode != MODE_5D);
    constexpr bool kAux = (kMode == MODE_S2 || kMode == MODE_S4);
    const int TS = a.tile, Ls = a.Ls;
    const int nthr = (TS * Ls + 31) / 32 * 32;
    const bool has_dot = (kMode == MODE_S4) && a.dot_part;
    const bool scale_bulk = (T::P == P16 || T::P == PFX16 || T::P == PFX8) && (Ls % 4 == 0);
    constexpr int KT = (LS > 0 && LS <= 8) ? 8 : 16;
    const StageSmem L = stage_smem(TS, Ls, T::NC, sizeof(LE), sizeof(R), kTma, kTC, scale_bulk, kAux,
                                   has_dot, !kTC || kMode == MODE_S4, KT, kMode != MODE_S4);
    static bool attr_set = false;
    if (!attr_set) {
        DWF_CUDA(cudaFuncSetAttribute(stage_kernel<T, kMode, kMphi, kStage, kDag, LS, TSC>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024));
        attr_set = true;
    }
    if (L.total > 220 * 1024) throw std::runtime_error("stage tile does not fit in shared memory");
    const long end = a.site_end ? a.site_end : a.nout;
    const long nblk = (end - a.site0) / TS;
    if (nblk <= 0) return;
    stage_kernel<T, kMode, kMphi, kStage, kDag, LS, TSC><<<(unsigned)nblk, nthr, L.total, st>>>(a);
    DWF_CUDA(cudaGetLastError());
    count_launch();
}

template <class T, bool kStage, int LS, int TSC>
static void dispatch_mode(StageMode mode, bool mphi, const StageArgs &a, cudaStream_t st)
{
    // the combinations the operators use: S1 (F, M_phi), S2, S3 (F, dagger),
    // S4 (dagger), and the fifth-dimension-only products
    if (mode == MODE_F && mphi && !a.dagger) launch_t<T, MODE_F, true, kStage, false, LS, TSC>(a, st);
    else if (mode == MODE_F && !mphi && a.dagger) launch_t<T, MODE_F, false, kStage, true, LS, TSC>(a, st);
    else if (mode == MODE_F && !mphi && !a.dagger) launch_t<T, MODE_F, false, kStage, false, LS, TSC>(a, st);
    else if (mode == MODE_S2 && !mphi && !a.dagger) launch_t<T, MODE_S2, false, kStage, false, LS, TSC>(a, st);
    else if (mode == MODE_S4 && !mphi && a.dagger) launch_t<T, MODE_S4, false, kStage, true, LS, TSC>(a, st);
    else if (mode == MODE_5D) launch_t<T, MODE_5D, false, false, false, LS, TSC>(a, st);
    else throw std::runtime_error("unsupported stage combination");
}

// Per-precision entry: compile-time fifth extent for Ls in {4, 8, 12, 16}
// with direct gathers, and a compile-time 8-site tile for Ls 8, 12 and 16 (the
// tile the autotuner picks on GB300); every other case (and bulk-copy
// gathers) uses the runtime-Ls, runtime-tile kernel.
template <class T>
void launch_stage_prec(StageMode mode, bool mphi, const StageArgs &a, cudaStream_t st)
{
    if constexpr (T::P != P64 && T::P != PFX8) {
        if (a.gather == 1) {
            dispatch_mode<T, true, 0, 0>(mode, mphi, a, st);
            return;
        }
    } else {
        if (a.gather == 1) throw std::runtime_error("no bulk-copy gather for this storage format");
    }
    if constexpr (T::P == P64) {
        // compile-time fifth extent for the reliable updates' common Ls
        if (a.Ls == 12) dispatch_mode<T, false, 12, 0>(mode, mphi, a, st);
        else if (a.Ls == 16) dispatch_mode<T, false, 16, 0>(mode, mphi, a, st);
        else dispatch_mode<T, false, 0, 0>(mode, mphi, a, st);
    } else {
        switch (a.Ls) {
        case 4: dispatch_mode<T, false, 4, 0>(mode, mphi, a, st); break;
        case 8:
            if (a.tile == 8) dispatch_mode<T, false, 8, 8>(mode, mphi, a, st);
            else dispatch_mode<T, false, 8, 0>(mode, mphi, a, st);
            break;
        case 12:
            if (a.tile == 8) dispatch_mode<T, false, 12, 8>(mode, mphi, a, st);
            else dispatch_mode<T, false, 12, 0>(mode, mphi, a, st);
            break;
        case 16:
            if (a.tile == 8) dispatch_mode<T, false, 16, 8>(mode, mphi, a, st);
            else dispatch_mode<T, false, 16, 0>(mode, mphi, a, st);
            break;
        default: dispatch_mode<T, false, 0, 0>(mode, mphi, a, st); break;
        }
    }
}

}  // namespace dwf
