// Device-side storage traits, loads/stores of packed 5D spinors and links,
// SU(3) reconstruction and the chiral-basis spin projectors of D^w.
#pragma once

#include "dwf_internal.h"

namespace dwf {

// ---------------------------------------------------------------- storage traits
struct TF64 {
    using R = double;
    static constexpr int NC = 12;   // 16-byte chunks per 5D site
    static constexpr Prec P = P64;
};
struct TF32 {
    using R = float;
    static constexpr int NC = 6;
    static constexpr Prec P = P32;
};
struct TF16 {
    using R = float;
    static constexpr int NC = 3;
    static constexpr Prec P = P16;
};
struct TBF16 {
    using R = float;
    static constexpr int NC = 3;
    static constexpr Prec P = PB16;
};
// 16-bit fixed point (Sec. 3.2): each real an int16, one FP32 scale per
// colour-spinor (the 24 reals of a (site, s)); the stored scale is
// max|v| / 32767, so value = integer * scale like the FP16 format
struct TFX16 {
    using R = float;
    static constexpr int NC = 3;
    static constexpr Prec P = PFX16;
};
constexpr float kFx16Max = 32767.f;
// 8-bit fixed point (Sec. 3.2, the paper's narrower fixed-point format): each
// real an int8, one FP32 scale per colour-spinor (stored max|v| / 127); the 24
// bytes of a (site, s) are three 8-byte chunks laid out [site][chunk][s][8 B],
// so a warp running over s still reads contiguous words
struct TFX8 {
    using R = float;
    static constexpr int NC = 3;
    static constexpr Prec P = PFX8;
};
constexpr float kFx8Max = 127.f;

// bytes of stored values per 5D site before the scale array
template <class T> __host__ __device__ constexpr int data_bytes() { return T::P == PFX8 ? 24 : 48; }

template <class T>
__device__ __forceinline__ const float *scale_ptr(const void *base, long nsite, int Ls)
{
    return reinterpret_cast<const float *>(reinterpret_cast<const char *>(base) +
                                           (size_t)nsite * Ls * data_bytes<T>());
}
template <class T>
__device__ __forceinline__ float *scale_ptr(void *base, long nsite, int Ls)
{
    return reinterpret_cast<float *>(reinterpret_cast<char *>(base) + (size_t)nsite * Ls * data_bytes<T>());
}

__device__ __forceinline__ void unpack8(const uint4 &u, float *v, __half)
{
    const __half2 *h = reinterpret_cast<const __half2 *>(&u);
#pragma unroll
    for (int i = 0; i < 4; i++) {
        float2 f = __half22float2(h[i]);
        v[2 * i] = f.x;
        v[2 * i + 1] = f.y;
    }
}
__device__ __forceinline__ void unpack8(const uint4 &u, float *v, __nv_bfloat16)
{
    const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&u);
#pragma unroll
    for (int i = 0; i < 4; i++) {
        float2 f = __bfloat1622float2(h[i]);
        v[2 * i] = f.x;
        v[2 * i + 1] = f.y;
    }
}
__device__ __forceinline__ uint4 pack8(const float *v, __half)
{
    uint4 u;
    __half2 *h = reinterpret_cast<__half2 *>(&u);
#pragma unroll
    for (int i = 0; i < 4; i++) h[i] = __floats2half2_rn(v[2 * i], v[2 * i + 1]);
    return u;
}
__device__ __forceinline__ uint4 pack8(const float *v, __nv_bfloat16)
{
    uint4 u;
    __nv_bfloat162 *h = reinterpret_cast<__nv_bfloat162 *>(&u);
#pragma unroll
    for (int i = 0; i < 4; i++) h[i] = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
    return u;
}

// Load the 24 reals of 5D site (site, s) of a packed field with nsite sites.
template <class T>
__device__ __forceinline__ void load_sp(const void *base, long nsite, long site, int s, int Ls,
                                        typename T::R *v);

template <>
__device__ __forceinline__ void load_sp<TF32>(const void *base, long, long site, int s, int Ls,
                                              float *v)
{
    const float4 *p = reinterpret_cast<const float4 *>(base) + (size_t)site * 6 * Ls + s;
#pragma unroll
    for (int c = 0; c < 6; c++) {
        float4 f = __ldg(p + (size_t)c * Ls);
        v[4 * c] = f.x;
        v[4 * c + 1] = f.y;
        v[4 * c + 2] = f.z;
        v[4 * c + 3] = f.w;
    }
}
template <>
__device__ __forceinline__ void load_sp<TF64>(const void *base, long, long site, int s, int Ls,
                                              double *v)
{
    const double2 *p = reinterpret_cast<const double2 *>(base) + (size_t)site * 12 * Ls + s;
#pragma unroll
    for (int c = 0; c < 12; c++) {
        double2 f = __ldg(p + (size_t)c * Ls);
        v[2 * c] = f.x;
        v[2 * c + 1] = f.y;
    }
}
template <>
__device__ __forceinline__ void load_sp<TBF16>(const void *base, long, long site, int s, int Ls,
                                               float *v)
{
    const uint4 *p = reinterpret_cast<const uint4 *>(base) + (size_t)site * 3 * Ls + s;
#pragma unroll
    for (int c = 0; c < 3; c++) unpack8(__ldg(p + (size_t)c * Ls), v + 8 * c, __nv_bfloat16());
}
// eight int16 of a 16-byte chunk to floats, without the conversion unit:
// with its sign bit flipped an int16 q reads as the unsigned q + 2^15, and
// the float whose bits are 0x4B000000 | (q + 2^15) is 2^23 + 2^15 + q exactly
constexpr float kFx16Bias = 8421376.f;  // 2^23 + 2^15
// the biased values 2^23 + 2^15 + q (exact integers below 2^24)
__device__ __forceinline__ void unpack8_fx16_biased(const uint4 &u, float *v)
{
    const uint32_t w[4] = {u.x ^ 0x80008000u, u.y ^ 0x80008000u, u.z ^ 0x80008000u, u.w ^ 0x80008000u};
#pragma unroll
    for (int i = 0; i < 4; i++) {
        v[2 * i] = __uint_as_float(__byte_perm(w[i], 0x4B00u, 0x5410));
        v[2 * i + 1] = __uint_as_float(__byte_perm(w[i], 0x4B00u, 0x5432));
    }
}
__device__ __forceinline__ void unpack8_fx16(const uint4 &u, float *v)
{
    unpack8_fx16_biased(u, v);
#pragma unroll
    for (int i = 0; i < 8; i++) v[i] -= kFx16Bias;
}
// eight floats times inv, each product within +-32767 (to a few ulp),
// rounded once to the nearest int16, ties to even: the fused v * inv +
// 1.5 * 2^23 rounds at the units place and leaves the integer, in two's
// complement, in the low 16 bits of the sum
__device__ __forceinline__ uint4 pack8_fx16(const float *v, float inv)
{
    constexpr float kRound = 12582912.f;  // 1.5 * 2^23
    uint32_t q[4];
#pragma unroll
    for (int i = 0; i < 4; i++)
        q[i] = __byte_perm(__float_as_uint(fmaf(v[2 * i], inv, kRound)),
                           __float_as_uint(fmaf(v[2 * i + 1], inv, kRound)), 0x5410);
    return make_uint4(q[0], q[1], q[2], q[3]);
}
// eight int8 of an 8-byte chunk to floats by bit placement: with its sign
// bit flipped an int8 q reads as the unsigned q + 128, and the float whose
// bits are 0x4B000000 | (q + 128) is 2^23 + 128 + q exactly
constexpr float kFx8Bias = 8388736.f;  // 2^23 + 128
__device__ __forceinline__ void unpack8_fx8(const uint2 &u, float *v)
{
    const uint32_t w[2] = {u.x ^ 0x80808080u, u.y ^ 0x80808080u};
#pragma unroll
    for (int i = 0; i < 2; i++)
#pragma unroll
        for (int b = 0; b < 4; b++)
            v[4 * i + b] = __uint_as_float(__byte_perm(w[i], 0x4B000000u, 0x7540u + b)) - kFx8Bias;
}
// eight floats times inv, each product within +-127 (to a few ulp), rounded
// once to the nearest int8 (ties to even) by the fused v * inv + 1.5 * 2^23,
// whose lowest byte is the integer in two's complement
__device__ __forceinline__ uint2 pack8_fx8(const float *v, float inv)
{
    constexpr float kRound = 12582912.f;  // 1.5 * 2^23
    uint32_t w[2];
#pragma unroll
    for (int i = 0; i < 2; i++) {
        const uint32_t f0 = __float_as_uint(fmaf(v[4 * i], inv, kRound));
        const uint32_t f1 = __float_as_uint(fmaf(v[4 * i + 1], inv, kRound));
        const uint32_t f2 = __float_as_uint(fmaf(v[4 * i + 2], inv, kRound));
        const uint32_t f3 = __float_as_uint(fmaf(v[4 * i + 3], inv, kRound));
        w[i] = __byte_perm(__byte_perm(f0, f1, 0x0040u), __byte_perm(f2, f3, 0x0040u), 0x5410u);
    }
    return make_uint2(w[0], w[1]);
}
template <>
__device__ __forceinline__ void load_sp<TFX8>(const void *base, long nsite, long site, int s, int Ls,
                                              float *v)
{
    const uint2 *p = reinterpret_cast<const uint2 *>(base) + (size_t)site * 3 * Ls + s;
#pragma unroll
    for (int c = 0; c < 3; c++) unpack8_fx8(__ldg(p + (size_t)c * Ls), v + 8 * c);
    const float sc = __ldg(scale_ptr<TFX8>(base, nsite, Ls) + (size_t)site * Ls + s);
#pragma unroll
    for (int i = 0; i < 24; i++) v[i] *= sc;
}

template <>
__device__ __forceinline__ void load_sp<TFX16>(const void *base, long nsite, long site, int s,
                                               int Ls, float *v)
{
    const uint4 *p = reinterpret_cast<const uint4 *>(base) + (size_t)site * 3 * Ls + s;
#pragma unroll
    for (int c = 0; c < 3; c++) unpack8_fx16(__ldg(p + (size_t)c * Ls), v + 8 * c);
    const float sc = __ldg(scale_ptr<TFX16>(base, nsite, Ls) + (size_t)site * Ls + s);
#pragma unroll
    for (int i = 0; i < 24; i++) v[i] *= sc;
}
template <>
__device__ __forceinline__ void load_sp<TF16>(const void *base, long nsite, long site, int s,
                                              int Ls, float *v)
{
    const uint4 *p = reinterpret_cast<const uint4 *>(base) + (size_t)site * 3 * Ls + s;
#pragma unroll
    for (int c = 0; c < 3; c++) unpack8(__ldg(p + (size_t)c * Ls), v + 8 * c, __half());
    const float sc = __ldg(scale_ptr<TF16>(base, nsite, Ls) + (size_t)site * Ls + s);
#pragma unroll
    for (int i = 0; i < 24; i++) v[i] *= sc;
}

template <class T>
__device__ __forceinline__ void store_sp(void *base, long nsite, long site, int s, int Ls,
                                         const typename T::R *v);

template <>
__device__ __forceinline__ void store_sp<TF32>(void *base, long, long site, int s, int Ls,
                                               const float *v)
{
    float4 *p = reinterpret_cast<float4 *>(base) + (size_t)site * 6 * Ls + s;
#pragma unroll
    for (int c = 0; c < 6; c++)
        p[(size_t)c * Ls] = make_float4(v[4 * c], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3]);
}
template <>
__device__ __forceinline__ void store_sp<TF64>(void *base, long, long site, int s, int Ls,
                                               const double *v)
{
    double2 *p = reinterpret_cast<double2 *>(base) + (size_t)site * 12 * Ls + s;
#pragma unroll
    for (int c = 0; c < 12; c++) p[(size_t)c * Ls] = make_double2(v[2 * c], v[2 * c + 1]);
}
template <>
__device__ __forceinline__ void store_sp<TBF16>(void *base, long, long site, int s, int Ls,
                                                const float *v)
{
    uint4 *p = reinterpret_cast<uint4 *>(base) + (size_t)site * 3 * Ls + s;
#pragma unroll
    for (int c = 0; c < 3; c++) p[(size_t)c * Ls] = pack8(v + 8 * c, __nv_bfloat16());
}
template <>
__device__ __forceinline__ void store_sp<TF16>(void *base, long nsite, long site, int s, int Ls,
                                               const float *v)
{
    float m = 0.f;
#pragma unroll
    for (int i = 0; i < 24; i++) m = fmaxf(m, fabsf(v[i]));
    const float sc = m > 0.f ? m : 1.f;
    const float inv = __fdividef(1.f, sc);  // stored value x scale = v to well within FP16 rounding
    float w[24];
#pragma unroll
    for (int i = 0; i < 24; i++) w[i] = v[i] * inv;
    uint4 *p = reinterpret_cast<uint4 *>(base) + (size_t)site * 3 * Ls + s;
#pragma unroll
    for (int c = 0; c < 3; c++) p[(size_t)c * Ls] = pack8(w + 8 * c, __half());
    scale_ptr<TF16>(base, nsite, Ls)[(size_t)site * Ls + s] = sc;
}

// 16-bit fixed-point store of v with the stored scale multiplied by f
__device__ __forceinline__ void store_fx16(void *base, long nsite, long site, int s, int Ls,
                                           const float *v, float f)
{
    float m = 0.f;
#pragma unroll
    for (int i = 0; i < 24; i++) m = fmaxf(m, fabsf(v[i]));
    const float sc = m > 0.f ? m / kFx16Max : 1.f;
    const float inv = m > 0.f ? kFx16Max / m : 0.f;
    // q = rint(v * inv) with the product exact; |v| <= m, so |v * inv|
    // exceeds 32767 by a few ulp at most and q stays within +-32767
    uint4 *p = reinterpret_cast<uint4 *>(base) + (size_t)site * 3 * Ls + s;
#pragma unroll
    for (int c = 0; c < 3; c++) p[(size_t)c * Ls] = pack8_fx16(v + 8 * c, inv);
    scale_ptr<TFX16>(base, nsite, Ls)[(size_t)site * Ls + s] = sc * f;
}
template <>
__device__ __forceinline__ void store_sp<TFX16>(void *base, long nsite, long site, int s, int Ls,
                                                const float *v)
{
    store_fx16(base, nsite, site, s, Ls, v, 1.f);
}

// 8-bit fixed-point store of v with the stored scale multiplied by f
__device__ __forceinline__ void store_fx8(void *base, long nsite, long site, int s, int Ls,
                                          const float *v, float f)
{
    float m = 0.f;
#pragma unroll
    for (int i = 0; i < 24; i++) m = fmaxf(m, fabsf(v[i]));
    const float sc = m > 0.f ? m / kFx8Max : 1.f;
    const float inv = m > 0.f ? kFx8Max / m : 0.f;
    uint2 *p = reinterpret_cast<uint2 *>(base) + (size_t)site * 3 * Ls + s;
#pragma unroll
    for (int c = 0; c < 3; c++) p[(size_t)c * Ls] = pack8_fx8(v + 8 * c, inv);
    scale_ptr<TFX8>(base, nsite, Ls)[(size_t)site * Ls + s] = sc * f;
}
template <>
__device__ __forceinline__ void store_sp<TFX8>(void *base, long nsite, long site, int s, int Ls,
                                               const float *v)
{
    store_fx8(base, nsite, site, s, Ls, v, 1.f);
}

// Scaled 16-bit store of v * f (FP16 or 16-bit fixed point): the values are
// normalised by max|v| and the factor goes into the stored scale only.
template <class T>
__device__ __forceinline__ void store_sp_scaled(void *base, long nsite, long site, int s, int Ls,
                                                const float *v, float f);
template <>
__device__ __forceinline__ void store_sp_scaled<TFX8>(void *base, long nsite, long site, int s, int Ls,
                                                      const float *v, float f)
{
    store_fx8(base, nsite, site, s, Ls, v, f);
}
template <>
__device__ __forceinline__ void store_sp_scaled<TFX16>(void *base, long nsite, long site, int s, int Ls,
                                                       const float *v, float f)
{
    store_fx16(base, nsite, site, s, Ls, v, f);
}
template <>
__device__ __forceinline__ void store_sp_scaled<TF16>(void *base, long nsite, long site, int s, int Ls,
                                                      const float *v, float f)
{
    float m = 0.f;
#pragma unroll
    for (int i = 0; i < 24; i++) m = fmaxf(m, fabsf(v[i]));
    const float sc = m > 0.f ? m : 1.f;
    const float inv = __fdividef(1.f, sc);  // stored value x scale = v to well within FP16 rounding
    float w[24];
#pragma unroll
    for (int i = 0; i < 24; i++) w[i] = v[i] * inv;
    uint4 *p = reinterpret_cast<uint4 *>(base) + (size_t)site * 3 * Ls + s;
#pragma unroll
    for (int c = 0; c < 3; c++) p[(size_t)c * Ls] = pack8(w + 8 * c, __half());
    scale_ptr<TF16>(base, nsite, Ls)[(size_t)site * Ls + s] = sc * f;
}

// ---------------------------------------------------------------- links
// Gathered link rows: [row][8 directions][12 reals] = rows 0 and 1 of the
// 3x3 complex matrix applied to the neighbour (U_{x,mu} forward,
// U^+_{x-mu,mu} backward).  Element type: double (F64), float (F32), half
// otherwise.
template <class T> struct LinkElem { using E = __half; };
template <> struct LinkElem<TF64> { using E = double; };
template <> struct LinkElem<TF32> { using E = float; };

template <class T>
__device__ __forceinline__ void load_link12(const void *links, long row, int k,
                                            typename T::R *u);
template <>
__device__ __forceinline__ void load_link12<TF32>(const void *links, long row, int k, float *u)
{
    const float4 *p = reinterpret_cast<const float4 *>(links) + ((size_t)row * 8 + k) * 3;
#pragma unroll
    for (int c = 0; c < 3; c++) {
        float4 f = __ldg(p + c);
        u[4 * c] = f.x;
        u[4 * c + 1] = f.y;
        u[4 * c + 2] = f.z;
        u[4 * c + 3] = f.w;
    }
}
template <>
__device__ __forceinline__ void load_link12<TF64>(const void *links, long row, int k, double *u)
{
    const double2 *p = reinterpret_cast<const double2 *>(links) + ((size_t)row * 8 + k) * 6;
#pragma unroll
    for (int c = 0; c < 6; c++) {
        double2 f = __ldg(p + c);
        u[2 * c] = f.x;
        u[2 * c + 1] = f.y;
    }
}
__device__ __forceinline__ void load_link12_half(const void *links, long row, int k, float *u)
{
    const uint2 *p = reinterpret_cast<const uint2 *>(links) + ((size_t)row * 8 + k) * 3;
#pragma unroll
    for (int c = 0; c < 3; c++) {
        uint2 w = __ldg(p + c);
        const __half2 *h = reinterpret_cast<const __half2 *>(&w);
        float2 a = __half22float2(h[0]), b = __half22float2(h[1]);
        u[4 * c] = a.x;
        u[4 * c + 1] = a.y;
        u[4 * c + 2] = b.x;
        u[4 * c + 3] = b.y;
    }
}
template <>
__device__ __forceinline__ void load_link12<TF16>(const void *links, long row, int k, float *u)
{
    load_link12_half(links, row, k, u);
}
template <>
__device__ __forceinline__ void load_link12<TBF16>(const void *links, long row, int k, float *u)
{
    load_link12_half(links, row, k, u);
}
template <>
__device__ __forceinline__ void load_link12<TFX16>(const void *links, long row, int k, float *u)
{
    load_link12_half(links, row, k, u);
}
template <>
__device__ __forceinline__ void load_link12<TFX8>(const void *links, long row, int k, float *u)
{
    load_link12_half(links, row, k, u);
}

// Third row of an SU(3) matrix: conj(row0 x row1).  u[18] = 3 rows x 3 cols x (re, im).
template <typename R>
__device__ __forceinline__ void reconstruct_row2(R *u)
{
#define RE(r, c) u[((r)*3 + (c)) * 2]
#define IM(r, c) u[((r)*3 + (c)) * 2 + 1]
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const int a = (c + 1) % 3, b = (c + 2) % 3;
        // z = row0[a] row1[b] - row0[b] row1[a]; row2[c] = conj(z)
        R zr = RE(0, a) * RE(1, b) - IM(0, a) * IM(1, b) - (RE(0, b) * RE(1, a) - IM(0, b) * IM(1, a));
        R zi = RE(0, a) * IM(1, b) + IM(0, a) * RE(1, b) - (RE(0, b) * IM(1, a) + IM(0, b) * RE(1, a));
        RE(2, c) = zr;
        IM(2, c) = -zi;
    }
#undef RE
#undef IM
}

// chi = U h for the two colour vectors of a half spinor, h[12] = [2][3][re,im].
template <typename R>
__device__ __forceinline__ void su3_mul_half(const R *u, const R *h, R *chi)
{
#pragma unroll
    for (int sp = 0; sp < 2; sp++)
#pragma unroll
        for (int r = 0; r < 3; r++) {
            R re = 0, im = 0;
#pragma unroll
            for (int c = 0; c < 3; c++) {
                const R ur = u[(r * 3 + c) * 2], ui = u[(r * 3 + c) * 2 + 1];
                const R hr = h[(sp * 3 + c) * 2], hi = h[(sp * 3 + c) * 2 + 1];
                re += ur * hr - ui * hi;
                im += ur * hi + ui * hr;
            }
            chi[(sp * 3 + r) * 2] = re;
            chi[(sp * 3 + r) * 2 + 1] = im;
        }
}

// Spin projection (1 + sg gamma_mu) psi -> half spinor h (chiral basis,
// gamma5 = diag(-1,-1,1,1)); then accumulation of the full spinor rebuilt from
// chi = U h.  psi/acc index (spin*3 + colour)*2 + reim.
//   mu=x: h0 = p0 + sg i p3, h1 = p1 + sg i p2; r2 = -sg i chi1, r3 = -sg i chi0
//   mu=y: h0 = p0 + sg p3,   h1 = p1 - sg p2;   r2 = -sg chi1,   r3 =  sg chi0
//   mu=z: h0 = p0 + sg i p2, h1 = p1 - sg i p3; r2 = -sg i chi0, r3 =  sg i chi1
//   mu=t: h0 = p0 + sg p2,   h1 = p1 + sg p3;   r2 =  sg chi0,   r3 =  sg chi1
template <typename R>
__device__ __forceinline__ void project(int mu, R sg, const R *p, R *h)
{
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const R p0r = p[(0 * 3 + c) * 2], p0i = p[(0 * 3 + c) * 2 + 1];
        const R p1r = p[(1 * 3 + c) * 2], p1i = p[(1 * 3 + c) * 2 + 1];
        const R p2r = p[(2 * 3 + c) * 2], p2i = p[(2 * 3 + c) * 2 + 1];
        const R p3r = p[(3 * 3 + c) * 2], p3i = p[(3 * 3 + c) * 2 + 1];
        R h0r, h0i, h1r, h1i;
        switch (mu) {
        case 0:  // + sg i p3 ; + sg i p2
            h0r = p0r - sg * p3i; h0i = p0i + sg * p3r;
            h1r = p1r - sg * p2i; h1i = p1i + sg * p2r;
            break;
        case 1:
            h0r = p0r + sg * p3r; h0i = p0i + sg * p3i;
            h1r = p1r - sg * p2r; h1i = p1i - sg * p2i;
            break;
        case 2:  // + sg i p2 ; - sg i p3
            h0r = p0r - sg * p2i; h0i = p0i + sg * p2r;
            h1r = p1r + sg * p3i; h1i = p1i - sg * p3r;
            break;
        default:
            h0r = p0r + sg * p2r; h0i = p0i + sg * p2i;
            h1r = p1r + sg * p3r; h1i = p1i + sg * p3i;
            break;
        }
        h[(0 * 3 + c) * 2] = h0r;
        h[(0 * 3 + c) * 2 + 1] = h0i;
        h[(1 * 3 + c) * 2] = h1r;
        h[(1 * 3 + c) * 2 + 1] = h1i;
    }
}

template <typename R>
__device__ __forceinline__ void accumulate(int mu, R sg, R w, const R *chi, R *acc)
{
    // w: overall factor (+1 or -1 from the boundary sign)
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const R c0r = w * chi[(0 * 3 + c) * 2], c0i = w * chi[(0 * 3 + c) * 2 + 1];
        const R c1r = w * chi[(1 * 3 + c) * 2], c1i = w * chi[(1 * 3 + c) * 2 + 1];
        acc[(0 * 3 + c) * 2] += c0r;
        acc[(0 * 3 + c) * 2 + 1] += c0i;
        acc[(1 * 3 + c) * 2] += c1r;
        acc[(1 * 3 + c) * 2 + 1] += c1i;
        R r2r, r2i, r3r, r3i;
        switch (mu) {
        case 0:  // r2 = -sg i c1 ; r3 = -sg i c0     (-i z = (z.i, -z.r))
            r2r = sg * c1i; r2i = -sg * c1r;
            r3r = sg * c0i; r3i = -sg * c0r;
            break;
        case 1:
            r2r = -sg * c1r; r2i = -sg * c1i;
            r3r = sg * c0r; r3i = sg * c0i;
            break;
        case 2:  // r2 = -sg i c0 ; r3 = sg i c1
            r2r = sg * c0i; r2i = -sg * c0r;
            r3r = -sg * c1i; r3i = sg * c1r;
            break;
        default:
            r2r = sg * c0r; r2i = sg * c0i;
            r3r = sg * c1r; r3i = sg * c1i;
            break;
        }
        acc[(2 * 3 + c) * 2] += r2r;
        acc[(2 * 3 + c) * 2 + 1] += r2i;
        acc[(3 * 3 + c) * 2] += r3r;
        acc[(3 * 3 + c) * 2 + 1] += r3i;
    }
}

}  // namespace dwf

namespace dwf {

// Compile-time variants of the projector and the rebuild-and-accumulate step:
// MU the direction, SG = +1 or -1 the sign in (1 + SG gamma_MU).  h is the
// half spinor, already multiplied by the neighbour's weight.  kBiased: p
// holds 16-bit fixed-point integers q as the exact floats 2^23 + 2^15 + q
// (unpack8_fx16_biased); a difference of two cancels the offset exactly and
// a sum takes it off once, a + (b - 2 offset), each step exact (integers
// below 2^24), so h is what the unbiased values give, with fewer operations.
template <int MU, int SG, typename R, bool kBiased = false>
__device__ __forceinline__ void project_ct(const R *p, R w, R *h)
{
    auto pl = [](R x, R y) {
        if constexpr (kBiased) return x + (y - R(2 * kFx16Bias));
        else return x + y;
    };
    auto mi = [](R x, R y) { return x - y; };
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const R p0r = p[(0 * 3 + c) * 2], p0i = p[(0 * 3 + c) * 2 + 1];
        const R p1r = p[(1 * 3 + c) * 2], p1i = p[(1 * 3 + c) * 2 + 1];
        const R p2r = p[(2 * 3 + c) * 2], p2i = p[(2 * 3 + c) * 2 + 1];
        const R p3r = p[(3 * 3 + c) * 2], p3i = p[(3 * 3 + c) * 2 + 1];
        R h0r, h0i, h1r, h1i;
        if constexpr (MU == 0) {  // h0 = p0 + SG i p3, h1 = p1 + SG i p2
            h0r = SG > 0 ? mi(p0r, p3i) : pl(p0r, p3i);
            h0i = SG > 0 ? pl(p0i, p3r) : mi(p0i, p3r);
            h1r = SG > 0 ? mi(p1r, p2i) : pl(p1r, p2i);
            h1i = SG > 0 ? pl(p1i, p2r) : mi(p1i, p2r);
        } else if constexpr (MU == 1) {  // h0 = p0 + SG p3, h1 = p1 - SG p2
            h0r = SG > 0 ? pl(p0r, p3r) : mi(p0r, p3r);
            h0i = SG > 0 ? pl(p0i, p3i) : mi(p0i, p3i);
            h1r = SG > 0 ? mi(p1r, p2r) : pl(p1r, p2r);
            h1i = SG > 0 ? mi(p1i, p2i) : pl(p1i, p2i);
        } else if constexpr (MU == 2) {  // h0 = p0 + SG i p2, h1 = p1 - SG i p3
            h0r = SG > 0 ? mi(p0r, p2i) : pl(p0r, p2i);
            h0i = SG > 0 ? pl(p0i, p2r) : mi(p0i, p2r);
            h1r = SG > 0 ? pl(p1r, p3i) : mi(p1r, p3i);
            h1i = SG > 0 ? mi(p1i, p3r) : pl(p1i, p3r);
        } else {  // h0 = p0 + SG p2, h1 = p1 + SG p3
            h0r = SG > 0 ? pl(p0r, p2r) : mi(p0r, p2r);
            h0i = SG > 0 ? pl(p0i, p2i) : mi(p0i, p2i);
            h1r = SG > 0 ? pl(p1r, p3r) : mi(p1r, p3r);
            h1i = SG > 0 ? pl(p1i, p3i) : mi(p1i, p3i);
        }
        h[(0 * 3 + c) * 2] = w * h0r;
        h[(0 * 3 + c) * 2 + 1] = w * h0i;
        h[(1 * 3 + c) * 2] = w * h1r;
        h[(1 * 3 + c) * 2 + 1] = w * h1i;
    }
}

template <int MU, int SG, typename R>
__device__ __forceinline__ void accumulate_ct(const R *chi, R *acc)
{
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const R c0r = chi[(0 * 3 + c) * 2], c0i = chi[(0 * 3 + c) * 2 + 1];
        const R c1r = chi[(1 * 3 + c) * 2], c1i = chi[(1 * 3 + c) * 2 + 1];
        acc[(0 * 3 + c) * 2] += c0r;
        acc[(0 * 3 + c) * 2 + 1] += c0i;
        acc[(1 * 3 + c) * 2] += c1r;
        acc[(1 * 3 + c) * 2 + 1] += c1i;
        R *a2 = acc + (2 * 3 + c) * 2, *a3 = acc + (3 * 3 + c) * 2;
        if constexpr (MU == 0) {  // r2 = -SG i c1 ; r3 = -SG i c0   (-i z = (z.i, -z.r))
            if (SG > 0) { a2[0] += c1i; a2[1] -= c1r; a3[0] += c0i; a3[1] -= c0r; }
            else        { a2[0] -= c1i; a2[1] += c1r; a3[0] -= c0i; a3[1] += c0r; }
        } else if constexpr (MU == 1) {  // r2 = -SG c1 ; r3 = SG c0
            if (SG > 0) { a2[0] -= c1r; a2[1] -= c1i; a3[0] += c0r; a3[1] += c0i; }
            else        { a2[0] += c1r; a2[1] += c1i; a3[0] -= c0r; a3[1] -= c0i; }
        } else if constexpr (MU == 2) {  // r2 = -SG i c0 ; r3 = SG i c1
            if (SG > 0) { a2[0] += c0i; a2[1] -= c0r; a3[0] -= c1i; a3[1] += c1r; }
            else        { a2[0] -= c0i; a2[1] += c0r; a3[0] += c1i; a3[1] -= c1r; }
        } else {  // r2 = SG c0 ; r3 = SG c1
            if (SG > 0) { a2[0] += c0r; a2[1] += c0i; a3[0] += c1r; a3[1] += c1i; }
            else        { a2[0] -= c0r; a2[1] -= c0i; a3[0] -= c1r; a3[1] -= c1i; }
        }
    }
}

// chi = U h reading U (3x3 complex, 20-real stride) from shared memory.
template <typename R>
__device__ __forceinline__ void su3_mul_half_smem(const R *U, const R *h, R *chi)
{
#pragma unroll
    for (int r = 0; r < 3; r++) {
        R u[6];
#pragma unroll
        for (int q = 0; q < 6; q++) u[q] = U[r * 6 + q];
#pragma unroll
        for (int sp = 0; sp < 2; sp++) {
            const R *hp = h + sp * 6;
            // complex dot product as a chain of fused multiply-adds
            R re = u[0] * hp[0];
            R im = u[0] * hp[1];
            re = fma(-u[1], hp[1], re);
            im = fma(u[1], hp[0], im);
#pragma unroll
            for (int c = 1; c < 3; c++) {
                re = fma(u[2 * c], hp[2 * c], re);
                im = fma(u[2 * c], hp[2 * c + 1], im);
                re = fma(-u[2 * c + 1], hp[2 * c + 1], re);
                im = fma(u[2 * c + 1], hp[2 * c], im);
            }
            chi[(sp * 3 + r) * 2] = re;
            chi[(sp * 3 + r) * 2 + 1] = im;
        }
    }
}

}  // namespace dwf
