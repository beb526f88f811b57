// Fused hop stage: one launch applies the Wilson hop D^w (or D^w^+) of
// Sec. 2.2 on one checkerboard, followed by the fifth-dimension matrices that
// follow it in Eq. (eq:detail) of Sec. 3.1.3, and optional axpy terms.
//
//   MODE_F : out = F . hop(in)
//   MODE_S2: y = aux - F . hop(in) ; out = G . y   (G null: out = y)
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
// Each F/G is an Ls x Ls real matrix per chirality, applied from shared
// memory.
//
// Thread mapping: a CTA owns `tile` output 4D sites and all Ls slices; thread
// (j, s) computes the hop of 5D site (j, s) into shared memory, then the dense
// fifth-dimension products read the whole Ls column of its site from there.
#include "device_common.cuh"

namespace dwf {

template <typename R>
struct Smem {
    R *F, *G, *H, *A;
    int hstride;  // reals per site in H/A (Ls*24 + 4 padding)
};

template <typename R>
__device__ __forceinline__ void load_mat_T(R *dst, const R *src, int Ls, int tid, int nthr)
{
    // dst[chi][t][s] = src[chi][s][t] (transposed so lanes with consecutive s hit
    // consecutive banks)
    const int n = 2 * Ls * Ls;
    for (int e = tid; e < n; e += nthr) {
        const int chi = e / (Ls * Ls), rem = e - chi * Ls * Ls;
        const int s = rem / Ls, t = rem - s * Ls;
        dst[(chi * Ls + t) * Ls + s] = src[e];
    }
}

// acc[r] (+)= sum_t M[chi(r)][s][t] X[site][t][r]
template <typename R, bool kAdd>
__device__ __forceinline__ void apply5(const R *MT, const R *X, int Ls, int s, R *acc, R coef)
{
    if (!kAdd) {
#pragma unroll
        for (int r = 0; r < 24; r++) acc[r] = 0;
    }
    for (int t = 0; t < Ls; t++) {
        const R f0 = coef * MT[(0 * Ls + t) * Ls + s];
        const R f1 = coef * MT[(1 * Ls + t) * Ls + s];
        const R *x = X + t * 24;
#pragma unroll
        for (int r = 0; r < 12; r++) acc[r] += f0 * x[r];
#pragma unroll
        for (int r = 12; r < 24; r++) acc[r] += f1 * x[r];
    }
}

template <class T, int kMode, bool kMphi>
__global__ void __launch_bounds__(512) stage_kernel(const StageArgs a)
{
    using R = typename T::R;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int Ls = a.Ls;
    const int tid = threadIdx.x;
    const int nthr = blockDim.x;
    const int jl = tid / Ls;
    const int s = tid - jl * Ls;
    const bool active = jl < a.tile;
    const long i = (long)blockIdx.x * a.tile + (active ? jl : 0);

    Smem<R> sm;
    sm.hstride = Ls * 24 + 4;
    sm.F = reinterpret_cast<R *>(smem_raw);
    sm.G = sm.F + 2 * Ls * Ls;
    sm.H = sm.G + 2 * Ls * Ls;
    sm.A = sm.H + a.tile * sm.hstride;

    const int sys = a.tile_sys ? a.tile_sys[((long)blockIdx.x * a.tile) / kSegPad] : 0;
    const R *Fg = reinterpret_cast<const R *>(a.F) + (size_t)sys * 2 * Ls * Ls;
    load_mat_T(sm.F, Fg, Ls, tid, nthr);
    if (a.G) load_mat_T(sm.G, reinterpret_cast<const R *>(a.G) + (size_t)sys * 2 * Ls * Ls, Ls, tid, nthr);

    const long seg = i / a.seg_out;
    const long loc = i - seg * a.seg_out;

    R acc[24];
#pragma unroll
    for (int r = 0; r < 24; r++) acc[r] = 0;

    if (kMode == MODE_5D) {
        if (active) load_sp<T>(a.in, a.nin, i, s, Ls, acc);
    } else if (active) {
        const long lrow = seg * a.link_stride + loc;
        R cb = 0, cc = 0, wm = 0;
        if (kMphi) {
            const double *mp = a.mphi + 3 * sys;
            cb = (R)(-0.5 * mp[0]);
            cc = (R)(-0.5 * mp[1]);
            wm = (R)(-mp[2]);
        }
#pragma unroll 1
        for (int k = 0; k < 8; k++) {
            const int e = __ldg(a.nbr + i * 8 + k);
            if (e == -1) continue;
            const long idx = e >= 0 ? e : (long)(-e - 2);
            const R w = e >= 0 ? R(1) : R(-1);
            const int mu = k >> 1;
            // forward (k even): 1 - gamma ; backward: 1 + gamma ; dagger flips
            const R sg = ((k & 1) ? R(1) : R(-1)) * (a.dagger ? R(-1) : R(1));
            R psi[24];
            load_sp<T>(a.in, a.nin, idx, s, Ls, psi);
            if (kMphi) {
                // (M_phi psi)_s = -(b psi_s + c (P_- psi_{s+1} + P_+ psi_{s-1}))/2,
                // wrap terms times -mass; P_- = spins 0,1, P_+ = spins 2,3
                R q[24];
                const int sp = s + 1 < Ls ? s + 1 : 0;
                const int sm1 = s > 0 ? s - 1 : Ls - 1;
                const R fp = s + 1 < Ls ? cc : cc * wm;
                const R fm = s > 0 ? cc : cc * wm;
                load_sp<T>(a.in, a.nin, idx, sp, Ls, q);
#pragma unroll
                for (int r = 0; r < 12; r++) psi[r] = cb * psi[r] + fp * q[r];
                load_sp<T>(a.in, a.nin, idx, sm1, Ls, q);
#pragma unroll
                for (int r = 12; r < 24; r++) psi[r] = cb * psi[r] + fm * q[r];
            }
            R h[12], chi[12], u[18];
            project<R>(mu, sg, psi, h);
            load_link12<T>(a.links, lrow, k, u);
            reconstruct_row2<R>(u);
            su3_mul_half<R>(u, h, chi);
            accumulate<R>(mu, sg, w, chi, acc);
        }
    }

    // hop result (or input, MODE_5D) to shared memory
    R *Hs = sm.H + jl * sm.hstride + s * 24;
    if (active) {
#pragma unroll
        for (int r = 0; r < 24; r++) Hs[r] = acc[r];
    }
    // own aux (MODE_S4 with G) to shared memory
    if (kMode == MODE_S4 && a.G && active) {
        R av[24];
        const long ai = seg * a.aux_stride + loc;
        load_sp<T>(a.aux, a.naux, ai, s, Ls, av);
        R *As = sm.A + jl * sm.hstride + s * 24;
#pragma unroll
        for (int r = 0; r < 24; r++) As[r] = av[r];
    }
    __syncthreads();

    R out[24];
    const R *Hsite = sm.H + jl * sm.hstride;
    if (kMode == MODE_F || kMode == MODE_5D) {
        if (active) apply5<R, false>(sm.F, Hsite, Ls, s, out, R(1));
    } else if (kMode == MODE_S2) {
        R y[24];
#pragma unroll
        for (int r = 0; r < 24; r++) y[r] = 0;
        if (active && loc < a.aux_valid) load_sp<T>(a.aux, a.naux, seg * a.aux_stride + loc, s, Ls, y);
        if (active) apply5<R, true>(sm.F, Hsite, Ls, s, y, R(-1));
        if (a.G) {
            R *As = sm.A + jl * sm.hstride + s * 24;
            if (active) {
#pragma unroll
                for (int r = 0; r < 24; r++) As[r] = y[r];
            }
            __syncthreads();
            if (active) apply5<R, false>(sm.G, sm.A + jl * sm.hstride, Ls, s, out, R(1));
        } else {
#pragma unroll
            for (int r = 0; r < 24; r++) out[r] = y[r];
        }
    } else {  // MODE_S4
        if (a.G) {
            if (active) apply5<R, false>(sm.G, sm.A + jl * sm.hstride, Ls, s, out, R(1));
        } else {
#pragma unroll
            for (int r = 0; r < 24; r++) out[r] = 0;
            if (active) load_sp<T>(a.aux, a.naux, seg * a.aux_stride + loc, s, Ls, out);
        }
        if (active) apply5<R, true>(sm.F, Hsite, Ls, s, out, R(-1));
    }

    if (active) store_sp<T>(a.out, a.nout, i, s, Ls, out);

    if (kMode == MODE_S4 && a.dot_part) {
        // partial <dotv, out> (real part), per-thread in R, across threads in FP64
        R d = 0;
        if (active) {
            R pv[24];
            load_sp<T>(a.dotv, a.nout, i, s, Ls, pv);
#pragma unroll
            for (int r = 0; r < 24; r++) d += pv[r] * out[r];
        }
        double dd = (double)d;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) dd += __shfl_xor_sync(0xffffffffu, dd, o);
        __shared__ double red[32];
        if ((tid & 31) == 0) red[tid >> 5] = dd;
        __syncthreads();
        if (tid < 32) {
            double v = tid < (nthr + 31) / 32 ? red[tid] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (tid == 0) a.dot_part[blockIdx.x] = v;
        }
    }
}

template <class T, int kMode, bool kMphi>
static void launch_t(const StageArgs &a, cudaStream_t st)
{
    using R = typename T::R;
    const int nthr = a.tile * a.Ls;
    const size_t smem = sizeof(R) * (4 * a.Ls * a.Ls + 2 * a.tile * (a.Ls * 24 + 4));
    static bool attr_set = false;
    if (!attr_set) {
        DWF_CUDA(cudaFuncSetAttribute(stage_kernel<T, kMode, kMphi>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
        attr_set = true;
    }
    const long nblk = a.nout / a.tile;
    stage_kernel<T, kMode, kMphi><<<(unsigned)nblk, nthr, smem, st>>>(a);
    DWF_CUDA(cudaGetLastError());
    count_launch();
}

template <class T>
static void dispatch_mode(StageMode mode, bool mphi, const StageArgs &a, cudaStream_t st)
{
    switch (mode) {
    case MODE_F:
        if (mphi) launch_t<T, MODE_F, true>(a, st);
        else launch_t<T, MODE_F, false>(a, st);
        break;
    case MODE_S2: launch_t<T, MODE_S2, false>(a, st); break;
    case MODE_S4: launch_t<T, MODE_S4, false>(a, st); break;
    case MODE_5D: launch_t<T, MODE_5D, false>(a, st); break;
    }
}

void launch_stage(Prec prec, StageMode mode, bool mphi_in, const StageArgs &a, cudaStream_t st)
{
    if (a.nout == 0) return;
    switch (prec) {
    case P64: dispatch_mode<TF64>(mode, mphi_in, a, st); break;
    case P32: dispatch_mode<TF32>(mode, mphi_in, a, st); break;
    case P16: dispatch_mode<TF16>(mode, mphi_in, a, st); break;
    case PB16: dispatch_mode<TBF16>(mode, mphi_in, a, st); break;
    }
}

}  // namespace dwf
