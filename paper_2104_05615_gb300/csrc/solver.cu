// Krylov drivers: preconditioned CG of Algorithm 1 with the multi-splitting
// preconditioner (Sec. 2.4: M = (+)_s A_s, a fixed number k of inner CG
// iterations from a zero guess, Sec. 2.5), Polak-Ribiere beta (Sec. 3.2),
// FP32 outer iterations with FP64 reliable updates (Sec. 3.2), and the
// optional reduced-Ls preconditioner of Sec. 3.3.
//
// Scalars (alpha, beta, <r,z>) live on the device per segment (system for
// the outer solve, block for the inner solves); the host reads only the
// residual norms to decide reliable updates and convergence.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <stdexcept>

#include "engine.h"

namespace dwf {

void launch_accum(void *x, void *xacc, Prec pacc, long nsite, int Ls, int tile, cudaStream_t st);

namespace {

constexpr int kBlasTile = 16;

// A piece of the iteration replayed as one CUDA graph.  The first run() with
// `use` captures the launches issued by f; later runs replay them.  Kernel
// counts follow the replays.
struct CapturedGraph {
    cudaGraphExec_t exec = nullptr;
    long long nkern = 0;
    CapturedGraph() = default;
    CapturedGraph(const CapturedGraph &) = delete;
    ~CapturedGraph()
    {
        if (exec) cudaGraphExecDestroy(exec);
    }
    template <class F>
    void run(cudaStream_t st, bool use, F &&f)
    {
        if (!use) {
            f();
            return;
        }
        if (!exec) {
            const long long c0 = launch_count();
            DWF_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
            try {
                f();
            } catch (...) {
                cudaGraph_t g = nullptr;
                cudaStreamEndCapture(st, &g);
                if (g) cudaGraphDestroy(g);
                throw;
            }
            cudaGraph_t g = nullptr;
            DWF_CUDA(cudaStreamEndCapture(st, &g));
            const cudaError_t e = cudaGraphInstantiate(&exec, g, 0);
            cudaGraphDestroy(g);
            DWF_CUDA(e);
            nkern = launch_count() - c0;
            count_launch(-nkern);  // captured, not yet run
        }
        DWF_CUDA(cudaGraphLaunch(exec, st));
        count_launch(nkern);
    }
};

// Arguments of a vector kernel; during a batched solve the engine's activity
// mask makes the CTAs of converged systems exit at once.
BlasArgs blas(const Engine &E, long nsite, int Ls, const uint16_t *tile_seg, double *part)
{
    BlasArgs a{};
    if (E.active) {
        a.tile_sys = E.tsys_e;
        a.active = E.active;
    }
    a.nsite = nsite;
    a.Ls = Ls;
    a.tile = kBlasTile;
    a.tile_seg = tile_seg;
    a.part = part;
    a.scal_sign[0] = a.scal_sign[1] = 1.0;
    return a;
}

ScalarArgs scal(const Seg &sg, const double *part, int ncomp, int sites_per_cta)
{
    ScalarArgs s{};
    s.part = part;
    s.ncomp = ncomp;
    s.tile_begin = sg.d_tile_begin;
    s.nseg = sg.nseg;
    s.sites_per_cta = sites_per_cta;
    return s;
}

struct Ctx {
    Engine &E;
    const dwf_solver_params &P;
    cudaStream_t st;
    long n;
    int Ls;
    int nsys;
    double *part;
};

// k iterations of CG, x0 = 0, on every block's local operator A_s at fifth
// extent L (Sec. 2.4, the inner solves), inner storage in P.inner_prec:
// z = CG_k((+)_s A_s) rhs.  rhs: packed, precision prhs, extent L (it may be
// the inner residual workspace itself); z: packed, precision pz, extent L.
// The blocks may be processed in waves (all k inner iterations of one wave
// before the next); the block-major site order makes every wave a contiguous
// site range.
static void inner_cg(Ctx &c, int L, const void *rhs, Prec prhs, void *z, Prec pz, int iters)
{
    Engine &E = c.E;
    const dwf_solver_params &P = c.P;
    const Prec pi = (Prec)P.inner_prec;
    const long n = c.n;
    void *rin = E.ws("in_r", field_bytes(pi, n, L));
    void *pin = E.ws("in_p", field_bytes(pi, n, L));
    void *Apin = E.ws("in_Ap", field_bytes(pi, n, L));
    void *zin = E.ws("in_z", field_bytes(P32, n, L));
    void *uin = E.ws("in_u", field_bytes(pi, n, L));  // M_phi p, written with p
    double *rr = E.ws_d("in_rr", E.nblk), *al = E.ws_d("in_al", E.nblk), *be = E.ws_d("in_be", E.nblk);
    const uint16_t *tsb = E.seg_blk.d_tile_seg;
    const double *mphi = E.mats(L).mphi;
    auto with_u = [&](BlasArgs &a) {
        a.mphi_out = uin;
        a.mphi_prec = pi;
        a.mphi = mphi;
        if (!a.tile_sys) a.tile_sys = E.tsys_e;
    };
    // the last inner update writes z itself (single precision path) unless
    // z is FP64; the first writes alpha p without reading z
    const bool z_direct = z != zin && pz != P64;
    const bool rhs_is_rin = rhs == rin;
    // default: every block in one wave (measured fastest on GB300: smaller,
    // L2-resident waves leave the latency-bound stages short of parallelism)
    const int wave = P.precond_wave > 0 ? std::min(P.precond_wave, E.nblk)
                     : P.precond_wave < 0 ? E.wave_blocks(pi, L) : E.nblk;
    for (int b0 = 0; b0 < E.nblk; b0 += wave) {
        const int b1 = std::min(E.nblk, b0 + wave);
        const long s0 = (long)b0 * E.Nb_pad, s1 = (long)b1 * E.Nb_pad;
        auto range = [&](BlasArgs &a) {
            a.site0 = s0;
            a.site_end = s1;
        };
        auto segs = [&](ScalarArgs &t) {
            t.seg0 = b0;
            t.nseg = b1 - b0;
        };
        {
            // p = r = rhs (inner precision), u = M_phi p, |r|^2 per block
            BlasArgs a = blas(E, n, L, tsb, c.part);
            range(a);
            a.v[0] = pin;
            a.p[0] = pi;
            a.v[1] = const_cast<void *>(rhs);
            a.p[1] = prhs;
            a.v[2] = rhs_is_rin ? nullptr : rin;
            a.p[2] = pi;
            with_u(a);
            launch_blas(BLAS_COPY, a, c.st);
            ScalarArgs t = scal(E.seg_blk, c.part, 1, kBlasTile);
            segs(t);
            t.s0 = rr;
            launch_scalar(SC_SUM, t, c.st);
        }
        for (int it = 0; it < iters; it++) {
            const bool last = it + 1 == iters;
            E.timed_begin(1 + it);
            const int tile = E.apply_local(pi, L, Apin, pin, c.part, b0, b1, uin);
            E.timed_end(1 + it);
            ScalarArgs t = scal(E.seg_blk, c.part, 1, tile);
            segs(t);
            t.s0 = rr;
            t.s1 = al;
            launch_scalar(SC_ALPHA, t, c.st);
            BlasArgs a = blas(E, n, L, tsb, (last && z_direct) ? nullptr : c.part);
            range(a);
            a.v[0] = zin; a.p[0] = P32;
            a.v[1] = pin; a.p[1] = pi;
            a.v[2] = rin; a.p[2] = pi;
            a.v[3] = Apin; a.p[3] = pi;
            a.scal[0] = al;
            a.x_zero = it == 0;
            if (last && z_direct) {
                a.v[4] = z; a.p[4] = pz;
                a.v[2] = a.v[3] = nullptr;
            }
            launch_blas(BLAS_CG_UPDATE, a, c.st);
            if (!last) {
                ScalarArgs u = scal(E.seg_blk, c.part, 1, kBlasTile);
                segs(u);
                u.s0 = rr;
                u.s1 = be;
                launch_scalar(SC_BETA_FR, u, c.st);
                BlasArgs x = blas(E, n, L, tsb, nullptr);
                range(x);
                x.v[0] = pin; x.p[0] = pi;
                x.v[1] = rin; x.p[1] = pi;
                x.scal[0] = be;
                with_u(x);
                launch_blas(BLAS_XPAY, x, c.st);
            }
        }
    }
    if (iters == 0) {
        BlasArgs a = blas(E, n, L, nullptr, nullptr);
        a.v[0] = z;
        a.p[0] = pz;
        launch_blas(BLAS_AXPY_ZERO, a, c.st);
    } else if (!z_direct && z != zin) {
        launch_convert(pz, z, P32, zin, n, L, c.st);
    }
}

// z = M^-1 r (outer precision po for r and z): the multi-splitting
// preconditioner, or its reduced-Ls form z = (T^+ Mhat^-1 T + mu) r (Sec. 3.3).
void precond_apply(Ctx &c, Prec po, const void *r, void *z, int &inner_count)
{
    Engine &E = c.E;
    const dwf_solver_params &P = c.P;
    const Prec pi = (Prec)P.inner_prec;
    const bool red = P.use_reduced_ls && E.Ls_hat > 0;
    const long n = c.n;
    if (red) {
        const int L = E.Ls_hat;
        void *rin = E.ws("in_r", field_bytes(pi, n, L));
        void *zin = E.ws("in_z", field_bytes(P32, n, L));
        // into BF16 (or 8-bit) inner storage the forward map runs on the tensor
        // cores with BF16 operands, the rounding of the storage it feeds; T^+
        // (FP32 output) stays in FP32 on the CUDA cores
        launch_tapply(pi, rin, L, po, r, E.Ls, E.Tm, n, 0, nullptr, P32, 0.0, c.st, true);
        inner_cg(c, L, rin, pi, zin, P32, P.inner_iters);
        launch_tapply(po, z, E.Ls, P32, zin, L, E.Tm, n, 1, r, po, E.mu, c.st);
    } else {
        inner_cg(c, E.Ls, r, po, z, po, P.inner_iters);
    }
    inner_count += P.inner_iters;
}

// r64 = b64 - A x64 ; r = r64 (in po) ; rr (per system) on the device
void true_residual(Ctx &c, Prec po, void *x64, const void *b64, void *Ax64, void *r64, void *r,
                   double *rr)
{
    c.E.apply_global(P64, DWF_OP_DDAGD, Ax64, x64, nullptr);
    BlasArgs a = blas(c.E, c.n, c.Ls, nullptr, c.part);
    a.v[0] = r64; a.p[0] = P64;
    a.v[1] = const_cast<void *>(b64); a.p[1] = P64;
    a.v[2] = Ax64; a.p[2] = P64;
    a.v[3] = (po != P64) ? r : nullptr; a.p[3] = po;
    launch_blas(BLAS_RESIDUAL, a, c.st);
    ScalarArgs s = scal(c.E.seg_sys, c.part, 1, kBlasTile);
    s.s0 = rr;
    launch_scalar(SC_SUM, s, c.st);
}

}  // namespace

dwf_status solve_impl(Engine &E, double *const *xs, const double *const *bs,
                      const dwf_solver_params &P, bool use_precond, SolveResult &res,
                      std::string &err);

dwf_status solve(Engine &E, double *const *xs, const double *const *bs, const dwf_solver_params &P,
                 bool use_precond, SolveResult &res, std::string &err)
{
    if (!P.use_graph) return solve_impl(E, xs, bs, P, use_precond, res, err);
    // graphs cannot be captured on the legacy default stream: run the solve on
    // the engine's own stream, ordered after and before the caller's stream
    const cudaStream_t user = E.st;
    if (!E.solve_stream) DWF_CUDA(cudaStreamCreateWithFlags(&E.solve_stream, cudaStreamNonBlocking));
    cudaEvent_t ev;
    DWF_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    DWF_CUDA(cudaEventRecord(ev, user));
    DWF_CUDA(cudaStreamWaitEvent(E.solve_stream, ev, 0));
    E.st = E.solve_stream;
    dwf_status s;
    try {
        s = solve_impl(E, xs, bs, P, use_precond, res, err);
    } catch (...) {
        E.st = user;
        cudaEventDestroy(ev);
        throw;
    }
    E.st = user;
    DWF_CUDA(cudaEventRecord(ev, E.solve_stream));
    DWF_CUDA(cudaStreamWaitEvent(user, ev, 0));
    cudaEventDestroy(ev);
    return s;
}

dwf_status solve_impl(Engine &E, double *const *xs, const double *const *bs,
                      const dwf_solver_params &P, bool use_precond, SolveResult &res,
                      std::string &err)
{
    const cudaStream_t st = E.st;
    const long n = E.ne;
    const int Ls = E.Ls;
    const int nsys = (int)E.sys.size();
    const Prec po = (Prec)P.outer_prec;
    // 16-bit outer vectors (the paper's 16-bit outer iterations, Sec. 3.2)
    // keep the solution increment in FP32 between reliable updates
    const Prec pacc = po == P64 ? P64 : P32;
    if (use_precond && (P.inner_prec == DWF_F64 || P.inner_iters < 0)) {
        err = "inner precision must be FP32, FP16, BF16 or FX16 and k >= 0";
        return DWF_EINVAL;
    }
    if (P.use_reduced_ls && use_precond && (E.Ls_hat <= 0 || !E.Tm)) {
        err = "reduced-Ls preconditioner requested but not configured";
        return DWF_EINVAL;
    }
    const long long launches0 = launch_count();
    // workspace: the max CTA count over all kernels is n sites / 8-site tiles (x2 components)
    const long max_cta = std::max<long>((long)E.nblk * E.E2_pad, n) / 4 + 16;
    Ctx c{E, P, st, n, Ls, nsys, E.ws_d("part", 2 * max_cta)};

    void *x64 = E.ws("x64", field_bytes(P64, n, Ls));
    void *b64 = E.ws("b64", field_bytes(P64, n, Ls));
    void *r64 = E.ws("r64", field_bytes(P64, n, Ls));
    void *Ax64 = E.ws("Ax64", field_bytes(P64, n, Ls));
    void *r = po == P64 ? r64 : E.ws("r_o", field_bytes(po, n, Ls));
    void *p = E.ws("p_o", field_bytes(po, n, Ls));
    void *Ap = E.ws("Ap_o", field_bytes(po, n, Ls));
    void *z = use_precond ? E.ws("z_o", field_bytes(po, n, Ls)) : r;
    void *xacc = po == P64 ? x64 : E.ws("xacc_o", field_bytes(pacc, n, Ls));
    void *u = E.ws("u_o", field_bytes(po, n, Ls));  // M_phi p, written with p
    const double *mphi_o = E.mats(Ls).mphi;
    auto with_u = [&](BlasArgs &a) {
        a.mphi_out = u;
        a.mphi_prec = po;
        a.mphi = mphi_o;
        if (!a.tile_sys) a.tile_sys = E.tsys_e;
    };
    double *bb = E.ws_d("bb", nsys), *rr = E.ws_d("rr", nsys), *rz = E.ws_d("rz", nsys);
    double *al = E.ws_d("al", nsys), *be = E.ws_d("be", nsys), *pAp = E.ws_d("pAp", nsys);

    EventPair ev;  // the solve's device time; destroyed on every exit path
    DWF_CUDA(cudaEventRecord(ev.e0, st));

    for (int k = 0; k < nsys; k++) {
        const LatticeGeom &g = *E.sys[k].g;
        launch_pack(P64, (char *)b64 + field_bytes(P64, E.sys[k].off, Ls), bs[k], E.perm[k], g.ne(),
                    g.Vh, Ls, st);
        launch_pack(P64, (char *)x64 + field_bytes(P64, E.sys[k].off, Ls), xs[k], E.perm[k], g.ne(),
                    g.Vh, Ls, st);
    }
    {
        BlasArgs a = blas(E, n, Ls, nullptr, c.part);
        a.v[0] = b64;
        a.p[0] = P64;
        launch_blas(BLAS_NORM2, a, st);
        ScalarArgs s = scal(E.seg_sys, c.part, 1, kBlasTile);
        s.s0 = bb;
        launch_scalar(SC_SUM, s, st);
    }
    std::vector<double> h_bb(nsys), h_rr(nsys), h_max(nsys), h_true(nsys);
    DWF_CUDA(cudaMemcpyAsync(h_bb.data(), bb, nsys * 8, cudaMemcpyDeviceToHost, st));
    true_residual(c, po, x64, b64, Ax64, r64, r, rr);
    if (po != P64) {
        BlasArgs a = blas(E, n, Ls, nullptr, nullptr);
        a.v[0] = xacc;
        a.p[0] = pacc;
        launch_blas(BLAS_AXPY_ZERO, a, st);
    }
    DWF_CUDA(cudaMemcpyAsync(h_rr.data(), rr, nsys * 8, cudaMemcpyDeviceToHost, st));
    DWF_CUDA(cudaStreamSynchronize(st));
    for (int k = 0; k < nsys; k++) {
        if (!(h_bb[k] > 0)) {
            err = "zero right-hand side";
            return DWF_EINVAL;
        }
        h_max[k] = h_rr[k];
    }
    const double tol2 = P.tol * P.tol;
    auto all_below = [&](const std::vector<double> &v) {
        for (int k = 0; k < nsys; k++)
            if (!(v[k] <= tol2 * h_bb[k])) return false;
        return true;
    };
    int inner_total = 0, ru = 0, iters = 0;
    // events around every operator application, from the first preconditioner on
    struct TimeScope {
        Engine &E;
        TimeScope(Engine &e, bool on) : E(e) { E.time_kernels = on; }
        ~TimeScope() { E.time_kernels = false; }
    } time_scope(E, P.time_kernels != 0 && P.precond_wave == 0);
    bool converged = all_below(h_rr);

    // p = z = M^-1 r ; rz = <r, z>
    if (!converged) {
        if (use_precond) {
            precond_apply(c, po, r, z, inner_total);
            E.timed_mark(1, P.inner_iters);
        }
        BlasArgs a = blas(E, n, Ls, E.seg_sys.d_tile_seg, c.part);
        a.v[0] = p; a.p[0] = po;
        a.v[1] = z; a.p[1] = po;
        with_u(a);
        launch_blas(BLAS_COPY, a, st);  // partial |z|^2 unused
        BlasArgs d = blas(E, n, Ls, nullptr, c.part);
        d.v[0] = r; d.p[0] = po;
        d.v[1] = z; d.p[1] = po;
        launch_blas(BLAS_DOT, d, st);
        ScalarArgs s = scal(E.seg_sys, c.part, 1, kBlasTile);
        s.s0 = rz;
        launch_scalar(SC_SUM, s, st);
    }
    const int maxiter = P.maxiter > 0 ? P.maxiter : 20000;
    const double delta2 = (P.delta > 0 ? P.delta : 0.1) * (P.delta > 0 ? P.delta : 0.1);
    // the two halves of an iteration; each becomes one CUDA graph after the
    // first (uncaptured) iteration has tuned and allocated everything
    double *h_rr_pin = E.pinned_d(nsys);
    auto half1 = [&]() {
        // alpha = <r,z> / <p, Ap> ; x += alpha p ; r -= alpha Ap ; |r|^2 to the host
        E.timed_begin(0);
        const int tile = E.apply_global(po, DWF_OP_DDAGD, Ap, p, c.part, nullptr, u);
        E.timed_end(0);
        {
            ScalarArgs s = scal(E.seg_sys, c.part, 1, tile);
            s.s0 = rz;
            s.s1 = al;
            s.s2 = pAp;
            launch_scalar(SC_ALPHA, s, st);
        }
        BlasArgs a = blas(E, n, Ls, E.seg_sys.d_tile_seg, c.part);
        a.v[0] = xacc; a.p[0] = pacc;
        a.v[1] = p; a.p[1] = po;
        a.v[2] = r; a.p[2] = po;
        a.v[3] = Ap; a.p[3] = po;
        a.scal[0] = al;
        launch_blas(BLAS_CG_UPDATE, a, st);
        ScalarArgs s = scal(E.seg_sys, c.part, 1, kBlasTile);
        s.s0 = rr;
        launch_scalar(SC_SUM, s, st);
        DWF_CUDA(cudaMemcpyAsync(h_rr_pin, rr, nsys * 8, cudaMemcpyDeviceToHost, st));
    };
    int inner_in_half2 = 0;
    auto half2 = [&]() {
        // z = M^-1 r ; beta ; p = z + beta p
        if (use_precond) {
            precond_apply(c, po, r, z, inner_in_half2);
            BlasArgs d = blas(E, n, Ls, nullptr, c.part);
            d.v[0] = z; d.p[0] = po;
            d.v[1] = r; d.p[1] = po;
            d.v[2] = Ap; d.p[2] = po;
            launch_blas(BLAS_DOT2, d, st);
            ScalarArgs s = scal(E.seg_sys, c.part, 2, kBlasTile);
            s.s0 = rz;
            s.s1 = al;
            s.s2 = be;
            launch_scalar(SC_BETA_PR, s, st);
        } else {
            BlasArgs d = blas(E, n, Ls, nullptr, c.part);
            d.v[0] = r; d.p[0] = po;
            launch_blas(BLAS_NORM2, d, st);
            ScalarArgs s = scal(E.seg_sys, c.part, 1, kBlasTile);
            s.s0 = rz;
            s.s1 = be;
            launch_scalar(SC_BETA_FR, s, st);
        }
        BlasArgs x = blas(E, n, Ls, E.seg_sys.d_tile_seg, nullptr);
        x.v[0] = p; x.p[0] = po;
        x.v[1] = z; x.p[1] = po;
        x.scal[0] = be;
        with_u(x);
        launch_blas(BLAS_XPAY, x, st);
    };
    // per-system activity (batches only): converged systems' CTAs exit at once
    std::vector<int> h_active(nsys, 1);
    int *d_active = nullptr;
    if (nsys > 1) {
        d_active = (int *)E.ws("active", nsys * sizeof(int));
        DWF_CUDA(cudaMemcpyAsync(d_active, h_active.data(), nsys * sizeof(int), cudaMemcpyHostToDevice, st));
        DWF_CUDA(cudaStreamSynchronize(st));
    }
    struct ActiveScope {
        Engine &E;
        ActiveScope(Engine &e, const int *a) : E(e) { E.active = a; }
        ~ActiveScope() { E.active = nullptr; }
    } active_scope(E, d_active);
    CapturedGraph g1, g2;
    double t_local = 0, t_outer = 0;
    long long n_local = 0, n_outer = 0;
    // the host reads |r|^2 (and decides reliable updates and convergence) only
    // every check_every iterations; in between the iterations are issued
    // back to back without a host synchronisation
    const int check_every = P.check_every > 1 ? P.check_every : 1;
    while (!converged && iters < maxiter) {
        const bool graph = P.use_graph && iters > 0;
        g1.run(st, graph, half1);
        E.timed_mark(0, 1);
        iters++;
        if (iters % check_every != 0 && iters < maxiter) {
            g2.run(st, graph, half2);
            if (use_precond) E.timed_mark(1, P.inner_iters);
            if (use_precond) inner_total += P.inner_iters;
            continue;
        }
        DWF_CUDA(cudaStreamSynchronize(st));
        // the previous preconditioner call and this outer operator have completed
        E.timed_collect(t_outer, n_outer, t_local, n_local);
        for (int k = 0; k < nsys; k++) h_rr[k] = h_rr_pin[k];
        for (int k = 0; k < nsys; k++)
            if (!std::isfinite(h_rr[k])) {
                err = "non-finite residual";
                return DWF_ENOCONV;
            }
        // per-system decisions (a batch freezes systems once verified)
        bool any_conv = false, changed = false;
        bool do_ru = false;
        for (int k = 0; k < nsys; k++) {
            if (!h_active[k]) continue;
            const bool ck = h_rr[k] <= tol2 * h_bb[k];
            any_conv |= ck;
            if (po == P64) {
                if (ck) {
                    h_active[k] = 0;
                    changed = true;
                }
            } else {
                h_max[k] = std::max(h_max[k], h_rr[k]);
                if (ck || h_rr[k] < delta2 * h_max[k]) do_ru = true;
            }
        }
        if (do_ru) {
            launch_accum(x64, xacc, pacc, n, Ls, kBlasTile, st);
            true_residual(c, po, x64, b64, Ax64, r64, r, rr);
            DWF_CUDA(cudaMemcpyAsync(h_rr.data(), rr, nsys * 8, cudaMemcpyDeviceToHost, st));
            DWF_CUDA(cudaStreamSynchronize(st));
            ru++;
            for (int k = 0; k < nsys; k++) {
                h_max[k] = h_rr[k];
                if (h_active[k] && any_conv && h_rr[k] <= tol2 * h_bb[k]) {
                    h_active[k] = 0;
                    changed = true;
                }
            }
        }
        if (changed) {
            int left = 0;
            for (int k = 0; k < nsys; k++) left += h_active[k];
            if (left == 0) {
                converged = true;
                break;
            }
            if (d_active) {
                DWF_CUDA(cudaMemcpyAsync(d_active, h_active.data(), nsys * sizeof(int),
                                         cudaMemcpyHostToDevice, st));
                DWF_CUDA(cudaStreamSynchronize(st));
            }
        }
        g2.run(st, graph, half2);
        if (use_precond) E.timed_mark(1, P.inner_iters);
        if (use_precond) inner_total += P.inner_iters;
    }
    // final solution and FP64 true residual (every system)
    E.active = nullptr;
    if (po != P64) launch_accum(x64, xacc, pacc, n, Ls, kBlasTile, st);
    true_residual(c, po, x64, b64, Ax64, r64, r, rr);
    for (int k = 0; k < nsys; k++) {
        const LatticeGeom &g = *E.sys[k].g;
        launch_unpack(P64, xs[k], (char *)x64 + field_bytes(P64, E.sys[k].off, Ls), E.perm[k],
                      g.ne(), g.Vh, Ls, st);
    }
    DWF_CUDA(cudaEventRecord(ev.e1, st));
    DWF_CUDA(cudaMemcpyAsync(h_rr.data(), rr, nsys * 8, cudaMemcpyDeviceToHost, st));
    DWF_CUDA(cudaStreamSynchronize(st));
    float ms = 0;
    DWF_CUDA(cudaEventElapsedTime(&ms, ev.e0, ev.e1));
    res.iters = iters;
    res.inner_total = inner_total;
    res.ru = ru;
    res.ms = ms;
    res.true_res.resize(nsys);
    bool ok = true;
    for (int k = 0; k < nsys; k++) {
        res.true_res[k] = std::sqrt(h_rr[k] / h_bb[k]);
        if (!(res.true_res[k] <= P.tol)) ok = false;
    }
    res.converged = ok;
    res.launches = launch_count() - launches0;
    E.timed_collect(t_outer, n_outer, t_local, n_local);
    res.local_ms = t_local;
    res.local_n = n_local;
    res.outer_ms = t_outer;
    res.outer_n = n_outer;
    if (E.check_err()) {
        err = "a bounded device wait gave up";
        return DWF_ETIMEOUT;
    }
    if (!ok) {
        err = "not converged within maxiter";
        return DWF_ENOCONV;
    }
    return DWF_OK;
}

// out = CG_iters(Mhat) in on canonical FP64 fields at the reduced extent
// (the "exact" Mhat^-1 of the transform training of Sec. 3.3).
void reduced_local_inverse(Engine &E, double *out, const double *in, int Ls_hat, int iters,
                           const dwf_solver_params &P)
{
    const long n = E.ne;
    Ctx c{E, P, E.st, n, Ls_hat, 1, E.ws_d("part", 2 * (std::max<long>((long)E.nblk * E.E2_pad, n) / 4 + 16))};
    void *in64 = E.ws("ri_in64", field_bytes(P64, n, Ls_hat));
    void *out32 = E.ws("ri_out32", field_bytes(P32, n, Ls_hat));
    const LatticeGeom &g = *E.sys[0].g;
    launch_pack(P64, in64, in, E.perm[0], g.ne(), g.Vh, Ls_hat, E.st);
    inner_cg(c, Ls_hat, in64, P64, out32, P32, iters);
    launch_convert(P64, in64, P32, out32, n, Ls_hat, E.st);  // (in64 reused for the result)
    launch_unpack(P64, out, in64, E.perm[0], g.ne(), g.Vh, Ls_hat, E.st);
}

void precondition_fp64(Engine &E, double *z, const double *r, const dwf_solver_params &P)
{
    const long n = E.ne;
    const int Ls = E.Ls;
    Ctx c{E, P, E.st, n, Ls, 1, E.ws_d("part", 2 * (std::max<long>((long)E.nblk * E.E2_pad, n) / 4 + 16))};
    void *r64 = E.ws("pc_r64", field_bytes(P64, n, Ls));
    void *r32 = E.ws("pc_r32", field_bytes(P32, n, Ls));
    void *z32 = E.ws("pc_z32", field_bytes(P32, n, Ls));
    const LatticeGeom &g = *E.sys[0].g;
    launch_pack(P64, r64, r, E.perm[0], g.ne(), g.Vh, Ls, E.st);
    launch_convert(P32, r32, P64, r64, n, Ls, E.st);
    int cnt = 0;
    precond_apply(c, P32, r32, z32, cnt);
    launch_convert(P64, r64, P32, z32, n, Ls, E.st);
    launch_unpack(P64, z, r64, E.perm[0], g.ne(), g.Vh, Ls, E.st);
}

}  // namespace dwf
