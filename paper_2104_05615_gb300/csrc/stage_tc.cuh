// Fused hop stage with the Wilson hop on the tensor cores (16-bit storage).
//
// The same stages as stage_kernel (MODE_F, MODE_S2, MODE_S4 of Eq. (eq:detail),
// Sec. 3.1.3), with the hop of Sec. 2.2 computed as a matrix product per
// output 4D site x:
//
//   hop[(spin, t), (c, re/im)] = sum over (k, c', re/im) of
//       phi_k[(spin, t), (c', re/im)] * U_k[(c', re/im), (c, re/im)]
//
// where k runs over the 8 neighbours (forward and backward in 4 directions),
// phi_k = [1; R_k] P_k psi_k is the neighbour's spinor at slice t projected
// with (1 -+ gamma_mu) and already rebuilt to four spins (R_k the 2x2 spin map
// that rebuilds spins 2, 3 from the half spinor), and U_k the 3x3 complex link
// applied to the neighbour, written as a real 6x6 block.  Per site this is
// M = 4 Ls rows (spin, slice), K = 8 directions x 8 (6 used), N = 8 (6 used):
// mma.sync m16n8k16 with FP16 operands and FP32 accumulation.  The links and
// the projected spinors are FP16 (the links are stored so); the sum over the
// eight directions and three colours runs in FP32 inside the tensor core.
//
// A CTA owns 8 output sites and all Ls slices; it has 8 warps.  Warp w first
// builds direction k = w of phi for all 8 sites (compile-time projector per
// warp), then, after a barrier, runs the products of site j = w.  Each
// neighbour's stored scale (per site and slice) enters phi as the ratio to
// the largest of the eight at that slice, so phi stays within [-2, 2]; the
// product is scaled back in FP32.  The fifth-dimension matrices that follow
// the hop are then applied exactly as in stage_kernel: [G | -F] on the
// tensor cores for MODE_F / MODE_S2, the bidiagonal M5op^+ / M_phi^+ on the
// CUDA cores for MODE_S4.  M_phi on load is not offered: the input of the
// first stage must be M_phi x already (the solvers write it with p).
#pragma once

#include "stage_impl.cuh"

namespace dwf {

constexpr int kTcSites = 8;               // output 4D sites per CTA, one warp each
constexpr int kTcThreads = 32 * kTcSites;
constexpr int kPhiRow = 72;               // halves per phi row: 8 directions x 8 + 8 (144 B,
                                          // an odd number of 16-byte units: ldmatrix
                                          // rows fall in distinct banks)

// Shared-memory layout of a tensor-core-hop stage CTA (byte offsets).
struct TcSmem {
    int nbr, U, ref, smax, bt, phi, total;
};
__host__ __device__ inline TcSmem tc_smem(int Ls, bool has_aux, bool fifth_tc)
{
    TcSmem m;
    int o = 0;
    m.nbr = o;
    o = align16(o + kTcSites * 8 * 4);
    m.U = o;
    o = align16(o + kTcSites * 8 * kLinkStride * 4);
    m.ref = o;
    o = align16(o + kTcSites * 16 * 4);
    m.smax = o;
    o = align16(o + kTcSites * 4);
    m.bt = o;
    o = align16(o + (fifth_tc ? (has_aux ? 2 : 1) * 2 * 16 * kTcRow(kTcSites) * 2 : 0));
    m.phi = o;
    // phi, later reused for the FP32 result D (fifth_tc) or the hop and aux
    // columns of the bidiagonal stage
    const int phi = kTcSites * 4 * Ls * kPhiRow * 2;
    const int epi = 2 * kTcSites * Ls * 24 * 4;
    o = align16(o + (phi > epi ? phi : epi));
    m.total = o;
    return m;
}


// Sixteen-byte ldmatrix of an m16n8k16 A fragment: lane l supplies row l % 16,
// column block l / 16 of the 16 x 16 tile at `base` (row pitch kPhiRow halves).
__device__ __forceinline__ void ldmatrix_x4(uint32_t addr, uint4 &r)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
                 : "r"(addr));
}

// Largest |value| of eight bfloat16 in a 16-byte chunk.
__device__ __forceinline__ float maxabs_bf16x8(const uint4 &u)
{
    const uint32_t w[4] = {u.x & 0x7FFF7FFFu, u.y & 0x7FFF7FFFu, u.z & 0x7FFF7FFFu, u.w & 0x7FFF7FFFu};
    // non-negative bfloat16 order like their bit patterns
    uint32_t m = 0;
#pragma unroll
    for (int q = 0; q < 4; q++) m = max(m, max(w[q] & 0xFFFFu, w[q] >> 16));
    return __uint_as_float(m << 16);
}

// The 24 stored values of a 5D spinor as 12 complex numbers in FP32, times f:
// FP16 (normalised halves), BF16 and 16-bit fixed point (integers).
template <class T>
__device__ __forceinline__ void decode24(const uint4 *raw, float f, float *v)
{
#pragma unroll
    for (int c = 0; c < 3; c++) {
        float q[8];
        if constexpr (T::P == PFX16) unpack8_fx16(raw[c], q);
        else if constexpr (T::P == P16) unpack8(raw[c], q, __half());
        else unpack8(raw[c], q, __nv_bfloat16());
#pragma unroll
        for (int e = 0; e < 8; e++) v[8 * c + e] = q[e] * f;
    }
}

// phi rows of one neighbour k = 2 mu + d at one slice: four spins x three
// colours (re, im) as half2 from the projected half spinor h[6] (already
// weighted): spins 0, 1 are h, spins 2, 3 are R h, with R from the
// reconstruction of the chiral basis (gamma5 = diag(-1, -1, 1, 1)):
//   mu=x: (-SG i h1, -SG i h0); mu=y: (-SG h1, SG h0);
//   mu=z: (-SG i h0, SG i h1);  mu=t: (SG h0, SG h1).
// Every operation on h here is exact (a sign or a swap of re and im).
template <int MU, int SG>
__device__ __forceinline__ void rebuild_rows(const __half2 *h, __half2 *r2, __half2 *r3)
{
    // i z = (-im, re); -i z = (im, -re)
    const __half2 ipos = __floats2half2_rn(-1.f, 1.f), ineg = __floats2half2_rn(1.f, -1.f);
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const __half2 h0 = h[c], h1 = h[3 + c];
        if constexpr (MU == 0) {
            r2[c] = __hmul2(swap_h2(h1), SG > 0 ? ineg : ipos);
            r3[c] = __hmul2(swap_h2(h0), SG > 0 ? ineg : ipos);
        } else if constexpr (MU == 1) {
            r2[c] = SG > 0 ? __hneg2(h1) : h1;
            r3[c] = SG > 0 ? h0 : __hneg2(h0);
        } else if constexpr (MU == 2) {
            r2[c] = __hmul2(swap_h2(h0), SG > 0 ? ineg : ipos);
            r3[c] = __hmul2(swap_h2(h1), SG > 0 ? ipos : ineg);
        } else {
            r2[c] = SG > 0 ? h0 : __hneg2(h0);
            r3[c] = SG > 0 ? h1 : __hneg2(h1);
        }
    }
}

// Projected half spinor (1 + SG gamma_MU) psi in FP32 (psi: 12 complex, spin-major).
template <int MU, int SG>
__device__ __forceinline__ void project_f32(const float *p, float *h)
{
    project_ct<MU, SG, float, false>(p, 1.f, h);
}

// Projected half spinor in half2 arithmetic from FP16 stored halves, times w.
template <int MU, int SG>
__device__ __forceinline__ void project_h2(const __half2 *p, __half2 w, __half2 *h)
{
    const __half2 ipos = __floats2half2_rn(-1.f, 1.f), ineg = __floats2half2_rn(1.f, -1.f);
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const __half2 p0 = p[c], p1 = p[3 + c], p2 = p[6 + c], p3 = p[9 + c];
        __half2 a, b;
        if constexpr (MU == 0) {  // h0 = p0 + SG i p3, h1 = p1 + SG i p2
            a = __hfma2(swap_h2(p3), SG > 0 ? ipos : ineg, p0);
            b = __hfma2(swap_h2(p2), SG > 0 ? ipos : ineg, p1);
        } else if constexpr (MU == 1) {  // h0 = p0 + SG p3, h1 = p1 - SG p2
            a = SG > 0 ? __hadd2(p0, p3) : __hsub2(p0, p3);
            b = SG > 0 ? __hsub2(p1, p2) : __hadd2(p1, p2);
        } else if constexpr (MU == 2) {  // h0 = p0 + SG i p2, h1 = p1 - SG i p3
            a = __hfma2(swap_h2(p2), SG > 0 ? ipos : ineg, p0);
            b = __hfma2(swap_h2(p3), SG > 0 ? ineg : ipos, p1);
        } else {  // h0 = p0 + SG p2, h1 = p1 + SG p3
            a = SG > 0 ? __hadd2(p0, p2) : __hsub2(p0, p2);
            b = SG > 0 ? __hadd2(p1, p3) : __hsub2(p1, p3);
        }
        h[c] = __hmul2(a, w);
        h[3 + c] = __hmul2(b, w);
    }
}

// Build direction K of phi for the CTA's sites from the gathered chunks:
// items (site j, slice t) over the warp's lanes.
template <class T, int K, bool kDag, int LS, int NROUND>
__device__ __forceinline__ void build_phi(const int *sN, const float *sRef, __half *phi_base, int lane,
                                          const float *sc, const uint4 (*raw)[3])
{
    constexpr int MU = K >> 1;
    constexpr int SG = ((K & 1) ? 1 : -1) * (kDag ? -1 : 1);
    constexpr int NITEM = kTcSites * LS;
    constexpr float kValMax = (T::P == PFX16) ? kFx16Max : 1.f;
#pragma unroll
    for (int r = 0; r < NROUND; r++) {
        const int it = r * 32 + lane;
        if (it >= NITEM) break;
        const int j = it / LS, t = it - j * LS;
        const int e = sN[j * 8 + K];
        uint4 row[4];  // spins 0..3: three colours (re, im) + one zero pair
        if (e == -1) {
#pragma unroll
            for (int q = 0; q < 4; q++) row[q] = make_uint4(0u, 0u, 0u, 0u);
        } else {
            const float ref = sRef[j * 16 + t];
            // weight of this neighbour relative to the slice's reference: its
            // stored scale over the reference (scaled formats), 1 / reference
            // for BF16, whose stored values are the values themselves
            const float num = (T::P == PB16) ? 1.f : sc[r];
            const float wgt = (e >= 0 ? 1.f : -1.f) * (ref > 0.f ? __fdividef(num, ref) : 0.f);
            __half2 h[6];
            if constexpr (T::P == P16) {
                project_h2<MU, SG>(reinterpret_cast<const __half2 *>(raw[r]), __float2half2_rn(wgt), h);
            } else {
                // BF16 values / their reference, fixed-point integers / 32767:
                // decoded and projected in FP32, one rounding to FP16
                float p[24], hf[12];
                decode24<T>(raw[r], 1.f, p);
                project_f32<MU, SG>(p, hf);
                const float f = wgt * (1.f / kValMax);
#pragma unroll
                for (int q = 0; q < 6; q++) h[q] = __floats2half2_rn(hf[2 * q] * f, hf[2 * q + 1] * f);
            }
            __half2 r2[3], r3[3];
            rebuild_rows<MU, SG>(h, r2, r3);
            row[0] = make_uint4(h2u(h[0]), h2u(h[1]), h2u(h[2]), 0u);
            row[1] = make_uint4(h2u(h[3]), h2u(h[4]), h2u(h[5]), 0u);
            row[2] = make_uint4(h2u(r2[0]), h2u(r2[1]), h2u(r2[2]), 0u);
            row[3] = make_uint4(h2u(r3[0]), h2u(r3[1]), h2u(r3[2]), 0u);
        }
        __half *phi = phi_base + (size_t)j * 4 * LS * kPhiRow;
#pragma unroll
        for (int q = 0; q < 4; q++)
            *reinterpret_cast<uint4 *>(phi + (size_t)(q * LS + t) * kPhiRow + K * 8) = row[q];
    }
}

// Gather pass of direction K: every (site, slice) item's neighbour spinor
// (raw 16-byte chunks, kept in registers) and its magnitude bound (stored
// scale for FP16 / fixed point, max-abs for BF16) into sc[]; the slice's
// running maximum over the eight directions into sRef.
template <class T, int K, int LS, int NROUND>
__device__ __forceinline__ void gather_pass(const StageArgs &a, const int *sN, float *sRef, int lane,
                                            float *sc, uint4 (*raw)[3])
{
    constexpr int NITEM = kTcSites * LS;
#pragma unroll
    for (int r = 0; r < NROUND; r++) {
        sc[r] = 0.f;
        const int it = r * 32 + lane;
        const int j = it / LS, t = it - j * LS;
        const int e = it < NITEM ? sN[j * 8 + K] : -1;
        if (e == -1) {
#pragma unroll
            for (int c = 0; c < 3; c++) raw[r][c] = make_uint4(0u, 0u, 0u, 0u);
            continue;
        }
        const long idx = e >= 0 ? (long)e : (long)(-e - 2);
        const uint4 *gp = reinterpret_cast<const uint4 *>(a.in) + (size_t)idx * 3 * LS + t;
#pragma unroll
        for (int c = 0; c < 3; c++) raw[r][c] = __ldg(gp + (size_t)c * LS);
        if constexpr (T::P != PB16) sc[r] = __ldg(scale_ptr<TF16>(a.in, a.nin, LS) + idx * LS + t);
    }
#pragma unroll
    for (int r = 0; r < NROUND; r++) {
        const int it = r * 32 + lane;
        if (it >= NITEM) break;
        const int j = it / LS, t = it - j * LS;
        if (sN[j * 8 + K] == -1) continue;
        if constexpr (T::P == PB16) {
#pragma unroll
            for (int c = 0; c < 3; c++) sc[r] = fmaxf(sc[r], maxabs_bf16x8(raw[r][c]));
        }
        atomicMax(reinterpret_cast<int *>(sRef + j * 16 + t), __float_as_int(sc[r]));
    }
}

template <class T, int kMode, bool kDag, int LS>
__global__ void __launch_bounds__(kTcThreads, 3) stage_tc_kernel(const StageArgs a)
{
    static_assert(LS % 4 == 0 && LS <= 16, "tensor-core hop needs Ls a multiple of 4, at most 16");
    constexpr int TS = kTcSites;
    constexpr bool kScale = (T::P == P16 || T::P == PFX16);
    constexpr bool kAux = (kMode == MODE_S2 || kMode == MODE_S4);
    constexpr bool kFifthTc = kMode != MODE_S4;
    constexpr int NMT = LS / 4;  // m-tiles of 16 rows (spin, slice)
    constexpr int NROUND = (TS * LS + 31) / 32;
    constexpr float kValMax = (T::P == PFX16) ? kFx16Max : 1.f;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const TcSmem L = tc_smem(LS, kAux, kFifthTc);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long i0 = a.site0 + (long)blockIdx.x * TS;
    const long cta = i0 / TS;
    const int sys = a.tile_sys ? a.tile_sys[i0 / kSegPad] : 0;
    if (a.active && !a.active[sys]) {
        if (kMode == MODE_S4 && a.dot_part && tid == 0) a.dot_part[cta] = 0.0;
        return;
    }
    int *sN = reinterpret_cast<int *>(smem_raw + L.nbr);
    float *sU = reinterpret_cast<float *>(smem_raw + L.U);
    float *sRef = reinterpret_cast<float *>(smem_raw + L.ref);
    float *sMax = reinterpret_cast<float *>(smem_raw + L.smax);
    __half *sPhi = reinterpret_cast<__half *>(smem_raw + L.phi);
    const int seg = (int)(i0 / a.seg_out);

    // ---- 1. neighbour indices and links of the tile (third row rebuilt)
    if (tid < TS * 8) {
        const int j = tid >> 3, k = tid & 7;
        const long ii = i0 + j;
        const long row = (long)seg * a.link_stride + (ii - (long)seg * a.seg_out);
        const int nb = __ldg(a.nbr + ii * 8 + k);
        sN[tid] = nb;
        float u[18];
        if (nb != -1) {
            load_link12<T>(a.links, row, k, u);
            reconstruct_row2<float>(u);
        } else {
#pragma unroll
            for (int q = 0; q < 18; q++) u[q] = 0.f;
        }
        float *dst = sU + tid * kLinkStride;
#pragma unroll
        for (int q = 0; q < 18; q++) dst[q] = u[q];
    }
    if (tid < TS * 16) sRef[tid] = 0.f;
    __syncthreads();

    // ---- 2. reference pass and phi: warp w handles direction k = w
    {
        float sc[NROUND];
        uint4 raw[NROUND][3];
        auto dir_switch = [&](auto f) {
            switch (warp) {
            case 0: f(std::integral_constant<int, 0>{}); break;
            case 1: f(std::integral_constant<int, 1>{}); break;
            case 2: f(std::integral_constant<int, 2>{}); break;
            case 3: f(std::integral_constant<int, 3>{}); break;
            case 4: f(std::integral_constant<int, 4>{}); break;
            case 5: f(std::integral_constant<int, 5>{}); break;
            case 6: f(std::integral_constant<int, 6>{}); break;
            default: f(std::integral_constant<int, 7>{}); break;
            }
        };
        dir_switch([&](auto kc) { gather_pass<T, decltype(kc)::value, LS, NROUND>(a, sN, sRef, lane, sc, raw); });
        __syncthreads();
        dir_switch([&](auto kc) {
            build_phi<T, decltype(kc)::value, kDag, LS, NROUND>(sN, sRef, sPhi, lane, sc, raw);
        });
    }
    __syncthreads();

    // ---- 3. hop products of site j = warp
    const int j = warp;
    const long i = i0 + j;
    const int loc = (int)(i - (long)seg * a.seg_out);
    const int g = lane >> 2, tg = lane & 3;
    float d[NMT][4];
    {
        // B fragments: K row (direction, c' = tg, re/im), N column g = (c, re/im)
        uint32_t bf[4][2];
        const int cc = g >> 1, ri = g & 1;
        const bool live = tg < 3 && g < 6;
#pragma unroll
        for (int q = 0; q < 4; q++)
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const int k = 2 * q + h;
                float ur = 0.f, ui = 0.f;
                if (live) {
                    const float2 u = *reinterpret_cast<const float2 *>(sU + (j * 8 + k) * kLinkStride +
                                                                       (cc * 3 + tg) * 2);
                    ur = u.x;
                    ui = u.y;
                }
                // out.re = Ur phi.re - Ui phi.im ; out.im = Ui phi.re + Ur phi.im
                bf[q][h] = ri == 0 ? pack_h2(ur, -ui) : pack_h2(ui, ur);
            }
        const __half *phi = sPhi + (size_t)j * 4 * LS * kPhiRow;
        const int arow = lane & 15, acol = (lane >> 4) * 8;
#pragma unroll
        for (int mt = 0; mt < NMT; mt++) {
#pragma unroll
            for (int e = 0; e < 4; e++) d[mt][e] = 0.f;
#pragma unroll
            for (int q = 0; q < 4; q++) {
                uint4 af;
                ldmatrix_x4(smem_u32(phi + (size_t)(mt * 16 + arow) * kPhiRow + q * 16 + acol), af);
                mma_16816(d[mt], af, bf[q][0], bf[q][1]);
            }
        }
    }
    // D row r = mt * 16 + g (+ 8) is (spin r / LS, slice r % LS); columns
    // 2 tg, 2 tg + 1 are colour tg (re, im) for tg < 3.  Scaled back to the
    // hop's value: times the slice reference (and 32767 for fixed point).
    {
        const float *ref = sRef + j * 16;
#pragma unroll
        for (int mt = 0; mt < NMT; mt++)
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const int r = mt * 16 + g + 8 * h;
                const float f = tg < 3 ? ref[r % LS] * kValMax : 0.f;
                d[mt][2 * h] *= f;
                d[mt][2 * h + 1] *= f;
            }
    }
    __syncthreads();  // every warp is done with phi: the region is reused below

    // epilogue threads: (site jl, slice s)
    const int jl = tid / LS, s = tid - jl * LS;
    const bool active = tid < TS * LS;
    const long ie = i0 + (active ? jl : 0);
    const int loce = (int)(ie - (long)seg * a.seg_out);
    float out[24];

    if constexpr (kMode == MODE_S4) {
        // ---------------------------------------------------------------
        // S4: out = M5op^+ aux - M_phi^+ h, both bidiagonal per chirality:
        // out = A aux + B P^T aux + (b h + c P^T h) / 2, (P^T v)_s = v_{s-1}
        // on spins 0, 1 and v_{s+1} on spins 2, 3, wrap terms times -mass
        float *sH = reinterpret_cast<float *>(smem_raw + L.phi);
        float *sA = sH + TS * LS * 24;
#pragma unroll
        for (int mt = 0; mt < NMT; mt++)
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const int r = mt * 16 + g + 8 * h;
                const int sp = r / LS, t = r - sp * LS;
                if (tg < 3)
                    *reinterpret_cast<float2 *>(sH + (j * LS + t) * 24 + sp * 6 + 2 * tg) =
                        make_float2(d[mt][2 * h], d[mt][2 * h + 1]);
            }
        float av[24];
        if (active) {
            load_sp<T>(a.aux, a.naux, (long)seg * a.aux_stride + loce, s, LS, av);
            store24(sA + (jl * LS + s) * 24, av);
        }
        __syncthreads();
        if (active) {
            const double *mp = a.mphi + 5 * sys;
            const float hb = (float)(0.5 * mp[0]), hc = (float)(0.5 * mp[1]), mass = (float)mp[2];
            const float cA = a.G ? (float)mp[3] : 1.f, cB = a.G ? (float)mp[4] : 0.f;
            const int sm = s > 0 ? s - 1 : LS - 1, sp = s + 1 < LS ? s + 1 : 0;
            const float flo = s > 0 ? 1.f : -mass, fhi = s + 1 < LS ? 1.f : -mass;
            const float *H0 = sH + (jl * LS + s) * 24;
            const float *Hm = sH + (jl * LS + sm) * 24, *Am = sA + (jl * LS + sm) * 24;
            const float *Hp = sH + (jl * LS + sp) * 24, *Ap = sA + (jl * LS + sp) * 24;
            const float bl = cB * flo, cl = hc * flo, bh = cB * fhi, ch = hc * fhi;
#pragma unroll
            for (int r = 0; r < 12; r++) out[r] = cA * av[r] + bl * Am[r] + hb * H0[r] + cl * Hm[r];
#pragma unroll
            for (int r = 12; r < 24; r++) out[r] = cA * av[r] + bh * Ap[r] + hb * H0[r] + ch * Hp[r];
            store_sp<T>(a.out, a.nout, ie, s, LS, out);
        }
        if (a.dot_part) {
            // partial <dotv, out> (real part), per thread in FP32, across threads in FP64
            float dsum = 0.f;
            if (active) {
                float pv[24];
                load_sp<T>(a.dotv, a.nout, ie, s, LS, pv);
#pragma unroll
                for (int r = 0; r < 24; r++) dsum += pv[r] * out[r];
            }
            double dd = (double)dsum;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) dd += __shfl_xor_sync(0xffffffffu, dd, o);
            __shared__ double red[kTcSites];
            if (lane == 0) red[warp] = dd;
            __syncthreads();
            if (tid == 0) {
                double v = 0.0;
#pragma unroll
                for (int w = 0; w < kTcSites; w++) v += red[w];
                a.dot_part[cta] = v;
            }
        }
    } else {
        // ---------------------------------------------------------------
        // tensor-core fifth-dimension product D = [G | -F] . [aux ; h] per
        // chirality (as stage_kernel), operands scaled by the site's max-abs
        constexpr int RS = kTcRow(TS);
        constexpr int nk = kAux ? 2 : 1;
        __half *sB = reinterpret_cast<__half *>(smem_raw + L.bt);
        // S2 reads aux only on the block interior, which comes first: a tile
        // beyond it has no aux (tiles never straddle the boundary)
        const bool aux_tile = kAux && (int)(i0 - (long)seg * a.seg_out) < a.aux_valid;
        if constexpr (LS < 16) {
            // slices LS..15 of every tile are zero (K padded to 16)
            constexpr int padq = (16 - LS) * RS / 8;
            for (int e = tid; e < nk * 2 * padq; e += kTcThreads) {
                const int tl = e / padq, q = e - tl * padq;
                reinterpret_cast<uint4 *>(sB + ((size_t)tl * 16 + LS) * RS)[q] = make_uint4(0u, 0u, 0u, 0u);
            }
        }
        // the aux column of site j: (slice, chunk) items over the lanes
        constexpr int NAUX = 3 * LS, NAR = (NAUX + 31) / 32;
        uint4 araw[NAR];
        float asc[NAR];
        float m = 0.f;
        if (kAux && aux_tile) {
            const long ai = (long)seg * a.aux_stride + loc;
#pragma unroll
            for (int r = 0; r < NAR; r++) {
                const int it = r * 32 + lane;
                araw[r] = make_uint4(0u, 0u, 0u, 0u);
                asc[r] = 0.f;
                if (it < NAUX) {
                    const int t = it / 3, c = it - 3 * t;
                    araw[r] = __ldg(reinterpret_cast<const uint4 *>(a.aux) + (size_t)ai * 3 * LS + (size_t)c * LS + t);
                    if constexpr (kScale) {
                        asc[r] = __ldg(scale_ptr<TF16>(a.aux, a.naux, LS) + ai * LS + t);
                        m = fmaxf(m, asc[r] * kValMax);
                    } else {
                        m = fmaxf(m, maxabs_bf16x8(araw[r]));
                    }
                }
            }
        }
#pragma unroll
        for (int mt = 0; mt < NMT; mt++)
#pragma unroll
            for (int e = 0; e < 4; e++) m = fmaxf(m, fabsf(d[mt][e]));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) sMax[j] = m;
        // any factor within a few ulp of 1/m keeps the FP16 operands in range
        const float inv = m > 0.f ? __fdividef(1.f, m) : 0.f;
        // hop -> tile nk - 1, row slice, column (site, spin % 2, colour, re/im)
        {
            __half *tile = sB + (size_t)(nk - 1) * 2 * 16 * RS;
#pragma unroll
            for (int mt = 0; mt < NMT; mt++)
#pragma unroll
                for (int h = 0; h < 2; h++) {
                    const int r = mt * 16 + g + 8 * h;
                    const int sp = r / LS, t = r - sp * LS;
                    if (tg < 3)
                        *reinterpret_cast<uint32_t *>(tile + ((size_t)(sp >> 1) * 16 + t) * RS + j * 12 +
                                                      (sp & 1) * 6 + 2 * tg) =
                            pack_h2(d[mt][2 * h] * inv, d[mt][2 * h + 1] * inv);
                }
        }
        // aux -> tile 0: chunk c holds halves 8c..8c+7 of the 24 (spin-major),
        // chirality 0 = halves 0..11, 1 = 12..23
        if (kAux && aux_tile) {
#pragma unroll
            for (int r = 0; r < NAR; r++) {
                const int it = r * 32 + lane;
                if (it >= NAUX) break;
                const int t = it / 3, c = it - 3 * t;
                uint32_t w[4];
                if constexpr (T::P == P16) {
                    const __half2 f2 = __float2half2_rn(asc[r] * inv);
                    const uint32_t *q = reinterpret_cast<const uint32_t *>(&araw[r]);
#pragma unroll
                    for (int e = 0; e < 4; e++) w[e] = h2u(__hmul2(u2h(q[e]), f2));
                } else {
                    float v[8];
                    if constexpr (T::P == PFX16) unpack8_fx16(araw[r], v);
                    else unpack8(araw[r], v, __nv_bfloat16());
                    const float f = kScale ? asc[r] * inv : inv;
#pragma unroll
                    for (int e = 0; e < 4; e++) w[e] = pack_h2(v[2 * e] * f, v[2 * e + 1] * f);
                }
                __half *row0 = sB + (size_t)t * RS + j * 12;              // chirality 0
                __half *row1 = sB + ((size_t)16 + t) * RS + j * 12;       // chirality 1
                if (c == 0) {
                    *reinterpret_cast<uint2 *>(row0) = make_uint2(w[0], w[1]);
                    *reinterpret_cast<uint2 *>(row0 + 4) = make_uint2(w[2], w[3]);
                } else if (c == 1) {
                    *reinterpret_cast<uint2 *>(row0 + 8) = make_uint2(w[0], w[1]);
                    *reinterpret_cast<uint2 *>(row1) = make_uint2(w[2], w[3]);
                } else {
                    *reinterpret_cast<uint2 *>(row1 + 4) = make_uint2(w[0], w[1]);
                    *reinterpret_cast<uint2 *>(row1 + 8) = make_uint2(w[2], w[3]);
                }
            }
        }
        __syncthreads();
        // units (chirality x pair of 8-column n-tiles), spread over the warps
        constexpr int npair = TS * 12 / 16;
        constexpr int nunit = 2 * npair;
        const uint4 *Af = reinterpret_cast<const uint4 *>(a.F) + (size_t)sys * 2 * 2 * 32;
        const int lr = (lane & 7) + 8 * ((lane >> 3) & 1);
        const int ln = 8 * (lane >> 4);
        float *sD = reinterpret_cast<float *>(smem_raw + L.phi);
        for (int u = warp; u < nunit; u += kTcSites) {
            const int chi = u / npair, pr = u - chi * npair;
            // A fragments [G | -F] of this chirality (fixed per system)
            uint4 af[nk];
#pragma unroll
            for (int kk = 0; kk < nk; kk++) af[kk] = __ldg(Af + ((chi * 2 + kk) * 32 + lane));
            float dd[8];
#pragma unroll
            for (int q = 0; q < 8; q++) dd[q] = 0.f;
#pragma unroll
            for (int kk = 0; kk < nk; kk++) {
                if (kAux && kk == 0 && !aux_tile) continue;  // no aux in this tile
                const __half *tb = sB + ((size_t)(kk * 2 + chi) * 16 + lr) * RS + pr * 16 + ln;
                uint32_t b0, b1, b2, b3;
                ldmatrix_x4_trans(smem_u32(tb), b0, b1, b2, b3);
                mma_16816(dd, af[kk], b0, b1);
                mma_16816(dd + 4, af[kk], b2, b3);
            }
            // D rows s = g, g + 8 ; columns 2 tg, 2 tg + 1 of each n-tile -> one site
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const int nd = pr * 16 + h * 8 + 2 * tg;
                const int jd = nd / 12, rd = chi * 12 + (nd - jd * 12);
                // the scaled formats fold the site scale into the stored scale
                const float sd = kScale ? 1.f : sMax[jd];
                if (g < LS)
                    *reinterpret_cast<float2 *>(sD + (jd * LS + g) * 24 + rd) =
                        make_float2(dd[4 * h] * sd, dd[4 * h + 1] * sd);
                if (g + 8 < LS)
                    *reinterpret_cast<float2 *>(sD + (jd * LS + g + 8) * 24 + rd) =
                        make_float2(dd[4 * h + 2] * sd, dd[4 * h + 3] * sd);
            }
        }
        __syncthreads();
        if (active) {
            const float4 *q4 = reinterpret_cast<const float4 *>(sD + (jl * LS + s) * 24);
#pragma unroll
            for (int c = 0; c < 6; c++) {
                const float4 f = q4[c];
                out[4 * c] = f.x;
                out[4 * c + 1] = f.y;
                out[4 * c + 2] = f.z;
                out[4 * c + 3] = f.w;
            }
            if constexpr (kScale) store_sp_scaled<T>(a.out, a.nout, ie, s, LS, out, sMax[jl]);
            else store_sp<T>(a.out, a.nout, ie, s, LS, out);
        }
    }
}

template <class T, int kMode, bool kDag, int LS>
static void launch_tc_t(const StageArgs &a, cudaStream_t st)
{
    constexpr bool kAux = (kMode == MODE_S2 || kMode == MODE_S4);
    const TcSmem L = tc_smem(LS, kAux, kMode != MODE_S4);
    static bool attr_set = false;
    if (!attr_set) {
        DWF_CUDA(cudaFuncSetAttribute(stage_tc_kernel<T, kMode, kDag, LS>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024));
        attr_set = true;
    }
    if (L.total > 220 * 1024) throw std::runtime_error("tensor-core stage does not fit in shared memory");
    const long end = a.site_end ? a.site_end : a.nout;
    if ((end - a.site0) % kTcSites || a.site0 % kTcSites)
        throw std::runtime_error("tensor-core stage: site range not a multiple of the tile");
    const long nblk = (end - a.site0) / kTcSites;
    if (nblk == 0) return;
    stage_tc_kernel<T, kMode, kDag, LS><<<(unsigned)nblk, kTcThreads, L.total, st>>>(a);
    DWF_CUDA(cudaGetLastError());
    count_launch();
}

template <class T, int LS>
static void dispatch_tc_mode(StageMode mode, bool mphi, const StageArgs &a, cudaStream_t st)
{
    if (mphi) throw std::runtime_error("tensor-core stage takes M_phi x precomputed");
    if (mode == MODE_F && !a.dagger) launch_tc_t<T, MODE_F, false, LS>(a, st);
    else if (mode == MODE_F && a.dagger) launch_tc_t<T, MODE_F, true, LS>(a, st);
    else if (mode == MODE_S2 && !a.dagger) launch_tc_t<T, MODE_S2, false, LS>(a, st);
    else if (mode == MODE_S4 && a.dagger) launch_tc_t<T, MODE_S4, true, LS>(a, st);
    else throw std::runtime_error("unsupported tensor-core stage combination");
}

// Entry for gather == 2 (16-bit storage, Ls in {4, 8, 12, 16}).
template <class T>
void launch_stage_tc(StageMode mode, bool mphi, const StageArgs &a, cudaStream_t st)
{
    switch (a.Ls) {
    case 4: dispatch_tc_mode<T, 4>(mode, mphi, a, st); break;
    case 8: dispatch_tc_mode<T, 8>(mode, mphi, a, st); break;
    case 12: dispatch_tc_mode<T, 12>(mode, mphi, a, st); break;
    case 16: dispatch_tc_mode<T, 16>(mode, mphi, a, st); break;
    default: throw std::runtime_error("tensor-core stage needs Ls in {4, 8, 12, 16}");
    }
}

}  // namespace dwf
