// extern "C" entry points declared in include/dwf.h.
#include <cstring>
#include <memory>
#include <new>
#include <stdexcept>
#include <string>
#include <vector>

#include "engine.h"

using namespace dwf;

struct dwf_handle {
    LatticeGeom g;
    std::vector<double> gauge;  // host canonical gauge (complex as double pairs)
    int Ls = 0;
    double b = 0, c = 0, M5 = 0, mass = 0;
    cudaStream_t st = 0;
    std::unique_ptr<Engine> E;
    std::string err;
    std::vector<float> T;
};

dwf::Engine *dwf_handle_engine(dwf_handle *h) { return h->E.get(); }
void dwf_handle_set_error(dwf_handle *h, const char *msg) { h->err = msg; }

struct dwf_batch {
    std::vector<dwf_handle *> hs;
    std::unique_ptr<Engine> E;
    std::string err;
};

namespace {

template <class F>
dwf_status guarded(std::string *err, F &&f)
{
    try {
        return f();
    } catch (const CudaError &e) {
        if (err) *err = std::string(e.what) + ": " + cudaGetErrorString(e.err);
        return e.err == cudaErrorMemoryAllocation ? DWF_ENOMEM : DWF_ECUDA;
    } catch (const std::bad_alloc &) {
        if (err) *err = "host allocation failed";
        return DWF_ENOMEM;
    } catch (const std::exception &e) {
        if (err) *err = e.what();
        return DWF_EINVAL;
    }
}

}  // namespace

extern "C" {

void dwf_default_params(dwf_solver_params *p)
{
    if (!p) return;
    p->tol = 1e-10;
    p->maxiter = 20000;
    p->inner_iters = 6;
    p->outer_prec = DWF_F32;
    p->inner_prec = DWF_F16;
    p->delta = 0.1;
    p->use_reduced_ls = 0;
    p->use_graph = 1;
    p->check_every = 1;
    p->time_kernels = 0;
    p->precond_wave = 0;
}

const char *dwf_status_string(dwf_status s)
{
    switch (s) {
    case DWF_OK: return "ok";
    case DWF_EINVAL: return "invalid argument";
    case DWF_ENOMEM: return "out of memory";
    case DWF_ECUDA: return "CUDA error";
    case DWF_ENOCONV: return "not converged";
    case DWF_ETIMEOUT: return "device wait timed out";
    case DWF_EUNSUPPORTED: return "unsupported";
    }
    return "unknown";
}

const char *dwf_last_error(const dwf_handle *h) { return h ? h->err.c_str() : "null handle"; }

dwf_status dwf_create(dwf_handle **out, const double *gauge_host, const int dims[4], int Ls,
                      double b, double c, double M5, double mass, const int subdomain[4],
                      int t_antiperiodic, void *cuda_stream)
{
    if (!out || !gauge_host || !dims) return DWF_EINVAL;
    *out = nullptr;
    if (Ls < 1 || Ls > 32) return DWF_EINVAL;
    std::unique_ptr<dwf_handle> h;
    try {
        h.reset(new dwf_handle());
    } catch (...) {
        return DWF_ENOMEM;
    }
    std::string err;
    if (!build_geometry(h->g, dims, subdomain, t_antiperiodic, err)) return DWF_EINVAL;
    if (h->g.nblk > 65535) return DWF_EUNSUPPORTED;
    h->Ls = Ls;
    h->b = b;
    h->c = c;
    h->M5 = M5;
    h->mass = mass;
    h->st = (cudaStream_t)cuda_stream;
    dwf_status s = guarded(&h->err, [&]() {
        h->gauge.assign(gauge_host, gauge_host + h->g.V * 4 * 18);
        h->E.reset(new Engine());
        SysInfo si;
        si.g = &h->g;
        si.gauge = h->gauge.data();
        si.mass = mass;
        h->E->init({si}, Ls, b, c, M5, h->st);
        return DWF_OK;
    });
    if (s != DWF_OK) return s;
    *out = h.release();
    return DWF_OK;
}

void dwf_destroy(dwf_handle *h) { delete h; }

size_t dwf_field_elems(const dwf_handle *h, int Ls)
{
    if (!h) return 0;
    return (size_t)(Ls > 0 ? Ls : h->Ls) * h->g.Vh * 12;
}

size_t dwf_packed_bytes(const dwf_handle *h, dwf_prec prec, int Ls)
{
    if (!h) return 0;
    return field_bytes((Prec)prec, h->E->ne, Ls > 0 ? Ls : h->Ls);
}

static void fill_geometry(const LatticeGeom &G, dwf_geometry *g)
{
    g->even_sites = G.Vh;
    g->even_sites_padded = G.ne();
    g->blocks = G.nblk;
    g->block_sites = G.Nb;
    g->block_sites_padded = G.Nb_pad;
    g->o1_sites = G.O1;
    g->o1_sites_padded = G.O1_pad;
    g->e2_sites = G.E2 - (G.Nb_pad - G.Nb);
    g->e2_sites_padded = G.E2_pad;
}

dwf_status dwf_get_geometry(const dwf_handle *h, dwf_geometry *g)
{
    if (!h || !g) return DWF_EINVAL;
    fill_geometry(h->g, g);
    return DWF_OK;
}

dwf_status dwf_query_geometry(const int dims[4], const int subdomain[4], dwf_geometry *g)
{
    if (!dims || !g) return DWF_EINVAL;
    try {
        LatticeGeom G;
        std::string err;
        if (!build_geometry(G, dims, subdomain, 0, err)) return DWF_EINVAL;
        if (G.nblk > 65535) return DWF_EUNSUPPORTED;
        fill_geometry(G, g);
    } catch (...) {
        return DWF_ENOMEM;
    }
    return DWF_OK;
}

static bool prec_ok(int p) { return p >= DWF_F64 && p <= DWF_FX8; }

dwf_status dwf_pack(dwf_handle *h, void *packed, const void *canon, dwf_prec prec, void *stream)
{
    if (!h || !packed || !canon || !prec_ok(prec)) return DWF_EINVAL;
    return guarded(&h->err, [&]() {
        StreamSwap sw(*h->E, stream);
        launch_pack((Prec)prec, packed, canon, h->E->perm[0], h->g.ne(), h->g.Vh, h->Ls, h->E->st);
        return DWF_OK;
    });
}

dwf_status dwf_unpack(dwf_handle *h, void *canon, const void *packed, dwf_prec prec, void *stream)
{
    if (!h || !packed || !canon || !prec_ok(prec)) return DWF_EINVAL;
    return guarded(&h->err, [&]() {
        StreamSwap sw(*h->E, stream);
        launch_unpack((Prec)prec, canon, packed, h->E->perm[0], h->g.ne(), h->g.Vh, h->Ls, h->E->st);
        return DWF_OK;
    });
}

static dwf_status apply_packed_impl(dwf_handle *h, void *out, const void *in, dwf_op op,
                                    dwf_prec prec)
{
    Engine &E = *h->E;
    switch (op) {
    case DWF_OP_D:
    case DWF_OP_DDAG:
    case DWF_OP_DDAGD: E.apply_global((Prec)prec, op, out, in, nullptr); break;
    case DWF_OP_LOCAL_DDAGD: E.apply_local((Prec)prec, E.Ls, out, in, nullptr); break;
    case DWF_OP_M5INV: E.apply_5d((Prec)prec, E.Ls, MK_M5I, out, in, E.ne); break;
    case DWF_OP_M5INVDAG: E.apply_5d((Prec)prec, E.Ls, MK_M5ID, out, in, E.ne); break;
    default: h->err = "unknown operator"; return DWF_EINVAL;
    }
    return DWF_OK;
}

dwf_status dwf_apply_packed(dwf_handle *h, void *out, const void *in, dwf_op op, dwf_prec prec,
                            void *stream)
{
    if (!h || !out || !in || !prec_ok(prec) || out == in) return DWF_EINVAL;
    return guarded(&h->err, [&]() {
        StreamSwap sw(*h->E, stream);
        return apply_packed_impl(h, out, in, op, prec);
    });
}

dwf_status dwf_apply(dwf_handle *h, void *out, const void *in, dwf_op op, dwf_prec prec,
                     void *stream)
{
    if (!h || !out || !in || !prec_ok(prec) || out == in) return DWF_EINVAL;
    return guarded(&h->err, [&]() {
        StreamSwap sw(*h->E, stream);
        Engine &E = *h->E;
        const size_t fb = field_bytes((Prec)prec, E.ne, h->Ls);
        void *pin = E.ws("api_in_" + std::to_string(prec), fb);
        void *pout = E.ws("api_out_" + std::to_string(prec), fb);
        launch_pack((Prec)prec, pin, in, E.perm[0], h->g.ne(), h->g.Vh, h->Ls, E.st);
        dwf_status s = apply_packed_impl(h, pout, pin, op, prec);
        if (s != DWF_OK) return s;
        launch_unpack((Prec)prec, out, pout, E.perm[0], h->g.ne(), h->g.Vh, h->Ls, E.st);
        if (E.check_err()) {
            h->err = "a bounded device wait gave up";
            return DWF_ETIMEOUT;
        }
        return DWF_OK;
    });
}

static dwf_status run_solve(dwf_handle *h, double *x, const double *b, const dwf_solver_params *p,
                            bool precond, dwf_stats *stats)
{
    if (!h || !x || !b) return DWF_EINVAL;
    dwf_solver_params P;
    if (p) P = *p;
    else dwf_default_params(&P);
    return guarded(&h->err, [&]() {
        SolveResult r;
        double *xs[1] = {x};
        const double *bs[1] = {b};
        dwf_status s = solve(*h->E, xs, bs, P, precond, r, h->err);
        if (stats) {
            stats->outer_iters = r.iters;
            stats->inner_iters_total = r.inner_total;
            stats->reliable_updates = r.ru;
            stats->converged = r.converged;
            stats->true_residual = r.true_res.empty() ? -1.0 : r.true_res[0];
            stats->time_total_ms = r.ms;
            stats->kernel_launches = r.launches;
            stats->local_op_ms = r.local_ms;
            stats->local_op_count = r.local_n;
            stats->outer_op_ms = r.outer_ms;
            stats->outer_op_count = r.outer_n;
        }
        return s;
    });
}

dwf_status dwf_cg(dwf_handle *h, double *x, const double *b, const dwf_solver_params *p,
                  dwf_stats *stats)
{
    return run_solve(h, x, b, p, false, stats);
}

dwf_status dwf_mspcg(dwf_handle *h, double *x, const double *b, const dwf_solver_params *p,
                     dwf_stats *stats)
{
    return run_solve(h, x, b, p, true, stats);
}

dwf_status dwf_solve_host(dwf_handle *h, double *x_host, const double *b_host,
                          const dwf_solver_params *p, int use_mspcg, dwf_stats *stats)
{
    if (!h || !x_host || !b_host) return DWF_EINVAL;
    return guarded(&h->err, [&]() {
        Engine &E = *h->E;
        const size_t bytes = dwf_field_elems(h, 0) * 16;
        double *xd = (double *)E.ws("host_x", bytes);
        double *bd = (double *)E.ws("host_b", bytes);
        DWF_CUDA(cudaMemcpyAsync(bd, b_host, bytes, cudaMemcpyHostToDevice, E.st));
        DWF_CUDA(cudaMemcpyAsync(xd, x_host, bytes, cudaMemcpyHostToDevice, E.st));
        dwf_status s = run_solve(h, xd, bd, p, use_mspcg != 0, stats);
        DWF_CUDA(cudaMemcpyAsync(x_host, xd, bytes, cudaMemcpyDeviceToHost, E.st));
        DWF_CUDA(cudaStreamSynchronize(E.st));
        return s;
    });
}

dwf_status dwf_precondition(dwf_handle *h, double *z, const double *r, const dwf_solver_params *p)
{
    if (!h || !z || !r) return DWF_EINVAL;
    dwf_solver_params P;
    if (p) P = *p;
    else dwf_default_params(&P);
    return guarded(&h->err, [&]() {
        precondition_fp64(*h->E, z, r, P);
        DWF_CUDA(cudaStreamSynchronize(h->E->st));
        return DWF_OK;
    });
}

dwf_status dwf_set_reduced_ls(dwf_handle *h, int Ls_hat, const double *T_host, double mu)
{
    if (!h || !T_host || Ls_hat < 1 || Ls_hat > 32) return DWF_EINVAL;
    return guarded(&h->err, [&]() {
        Engine &E = *h->E;
        const size_t n = (size_t)4 * Ls_hat * 4 * h->Ls * 2;
        h->T.assign(T_host, T_host + n);
        float *d = (float *)E.ws("T_matrix", n * sizeof(float));
        DWF_CUDA(cudaMemcpy(d, h->T.data(), n * sizeof(float), cudaMemcpyHostToDevice));
        E.Tm = d;
        E.Ls_hat = Ls_hat;
        E.mu = mu;
        return DWF_OK;
    });
}

dwf_status dwf_reduced_local_inverse(dwf_handle *h, double *out, const double *in, int Ls_hat, int iters,
                                     const dwf_solver_params *p)
{
    if (!h || !out || !in || out == in || Ls_hat < 1 || Ls_hat > 32 || iters < 0) return DWF_EINVAL;
    dwf_solver_params P;
    if (p) P = *p;
    else dwf_default_params(&P);
    if (!prec_ok(P.inner_prec) || P.inner_prec == DWF_F64) return DWF_EINVAL;
    if (P.inner_prec >= DWF_F16 && Ls_hat > 16) return DWF_EINVAL;
    return guarded(&h->err, [&]() {
        reduced_local_inverse(*h->E, out, in, Ls_hat, iters, P);
        DWF_CUDA(cudaStreamSynchronize(h->E->st));
        if (h->E->check_err()) {
            h->err = "a bounded device wait gave up";
            return DWF_ETIMEOUT;
        }
        return DWF_OK;
    });
}

dwf_status dwf_apply_T(dwf_handle *h, double *out, const double *in, const double *T_host, int Ls_hat,
                       int dagger)
{
    if (!h || !out || !in || !T_host || out == in || Ls_hat < 1 || Ls_hat > 32) return DWF_EINVAL;
    return guarded(&h->err, [&]() {
        Engine &E = *h->E;
        const int Ls = h->Ls;
        const long n = E.ne;
        const size_t nT = (size_t)4 * Ls_hat * 4 * Ls * 2;
        std::vector<float> Tf(T_host, T_host + nT);
        float *Td = (float *)E.ws("T_apply_matrix", nT * sizeof(float));
        DWF_CUDA(cudaMemcpyAsync(Td, Tf.data(), nT * sizeof(float), cudaMemcpyHostToDevice, E.st));
        const int Lin = dagger ? Ls_hat : Ls, Lout = dagger ? Ls : Ls_hat;
        void *pin = E.ws("T_apply_in", field_bytes(P64, n, Lin));
        void *pout = E.ws("T_apply_out", field_bytes(P64, n, Lout));
        const LatticeGeom &g = *E.sys[0].g;
        launch_pack(P64, pin, in, E.perm[0], g.ne(), g.Vh, Lin, E.st);
        launch_tapply(P64, pout, Lout, P64, pin, Lin, Td, n, dagger ? 1 : 0, nullptr, P64, 0.0, E.st);
        launch_unpack(P64, out, pout, E.perm[0], g.ne(), g.Vh, Lout, E.st);
        DWF_CUDA(cudaStreamSynchronize(E.st));
        return DWF_OK;
    });
}

dwf_status dwf_T_contract(dwf_handle *h, double *G_host, const double *a, int La, const double *b, int Lb)
{
    if (!h || !G_host || !a || !b || La < 1 || Lb < 1 || 16 * La * Lb > 4096) return DWF_EINVAL;
    return guarded(&h->err, [&]() {
        Engine &E = *h->E;
        const size_t nG = (size_t)16 * La * Lb * 2;
        double *Gd = (double *)E.ws("T_contract_G", nG * sizeof(double));
        void *work = E.ws("T_contract_work", tcontract_workspace_bytes(La, Lb));
        const LatticeGeom &g = *E.sys[0].g;
        launch_tcontract(Gd, a, La, b, Lb, g.Vh, work, E.st);
        DWF_CUDA(cudaMemcpyAsync(G_host, Gd, nG * sizeof(double), cudaMemcpyDeviceToHost, E.st));
        DWF_CUDA(cudaStreamSynchronize(E.st));
        return DWF_OK;
    });
}

static bool field_prec(int p) { return p == DWF_F64 || p == DWF_F32; }

dwf_status dwf_field_axpby(dwf_handle *h, void *out, dwf_prec out_prec, double a_re, double a_im, const void *x,
                           double b_re, double b_im, const void *y, dwf_prec in_prec, int Ls)
{
    if (!h || !out || !x || !field_prec(out_prec) || !field_prec(in_prec) || Ls < 0 || Ls > 32) return DWF_EINVAL;
    return guarded(&h->err, [&]() {
        const long n = (long)dwf_field_elems(h, Ls);
        launch_field_axpby(out, (Prec)out_prec, x, y, (Prec)in_prec, a_re, a_im, b_re, b_im, n, h->E->st);
        DWF_CUDA(cudaStreamSynchronize(h->E->st));
        return DWF_OK;
    });
}

dwf_status dwf_field_dot(dwf_handle *h, double *result_host, const void *a, const void *b, dwf_prec prec, int Ls)
{
    if (!h || !result_host || !a || !b || !field_prec(prec) || Ls < 0 || Ls > 32) return DWF_EINVAL;
    return guarded(&h->err, [&]() {
        Engine &E = *h->E;
        const long n = (long)dwf_field_elems(h, Ls);
        void *work = E.ws("field_dot_work", field_dot_workspace_bytes());
        double *res = (double *)E.ws("field_dot_result", 2 * sizeof(double));
        launch_field_dot(res, a, b, (Prec)prec, n, work, E.st);
        DWF_CUDA(cudaMemcpyAsync(result_host, res, 2 * sizeof(double), cudaMemcpyDeviceToHost, E.st));
        DWF_CUDA(cudaStreamSynchronize(E.st));
        return DWF_OK;
    });
}

dwf_status dwf_set_local_truncated(dwf_handle *h, int on)
{
    if (!h) return DWF_EINVAL;
    return guarded(&h->err, [&]() {
        h->E->set_local_truncated(on != 0);
        return DWF_OK;
    });
}

dwf_status dwf_batch_create(dwf_batch **out, dwf_handle *const *hs, int n)
{
    if (!out || !hs || n < 1) return DWF_EINVAL;
    *out = nullptr;
    std::unique_ptr<dwf_batch> bt(new (std::nothrow) dwf_batch());
    if (!bt) return DWF_ENOMEM;
    for (int k = 0; k < n; k++) {
        if (!hs[k]) return DWF_EINVAL;
        if (hs[k]->Ls != hs[0]->Ls || hs[k]->b != hs[0]->b || hs[k]->c != hs[0]->c ||
            hs[k]->M5 != hs[0]->M5)
            return DWF_EINVAL;
        bt->hs.push_back(hs[k]);
    }
    dwf_status s = guarded(&bt->err, [&]() {
        std::vector<SysInfo> sv;
        for (auto *h : bt->hs) {
            SysInfo si;
            si.g = &h->g;
            si.gauge = h->gauge.data();
            si.mass = h->mass;
            sv.push_back(si);
        }
        bt->E.reset(new Engine());
        bt->E->init(sv, hs[0]->Ls, hs[0]->b, hs[0]->c, hs[0]->M5, hs[0]->st);
        return DWF_OK;
    });
    if (s != DWF_OK) return s;
    *out = bt.release();
    return DWF_OK;
}

void dwf_batch_destroy(dwf_batch *bt) { delete bt; }

dwf_status dwf_batch_mspcg(dwf_batch *bt, double *const *xs, const double *const *bs,
                           const dwf_solver_params *p, dwf_stats *per_system, dwf_stats *total)
{
    if (!bt || !xs || !bs) return DWF_EINVAL;
    dwf_solver_params P;
    if (p) P = *p;
    else dwf_default_params(&P);
    return guarded(&bt->err, [&]() {
        SolveResult r;
        dwf_status s = solve(*bt->E, xs, bs, P, true, r, bt->err);
        const int n = (int)bt->hs.size();
        if (per_system)
            for (int k = 0; k < n; k++) {
                per_system[k].outer_iters = r.iters;
                per_system[k].inner_iters_total = r.inner_total;
                per_system[k].reliable_updates = r.ru;
                per_system[k].true_residual = r.true_res.empty() ? -1 : r.true_res[k];
                per_system[k].converged = r.true_res.empty() ? 0 : r.true_res[k] <= P.tol;
                per_system[k].time_total_ms = r.ms;
                per_system[k].kernel_launches = r.launches;
            }
        if (total) {
            total->outer_iters = r.iters;
            total->inner_iters_total = r.inner_total;
            total->reliable_updates = r.ru;
            total->converged = r.converged;
            double mx = 0;
            for (double v : r.true_res) mx = v > mx ? v : mx;
            total->true_residual = mx;
            total->time_total_ms = r.ms;
            total->kernel_launches = r.launches;
            total->local_op_ms = r.local_ms;
            total->local_op_count = r.local_n;
            total->outer_op_ms = r.outer_ms;
            total->outer_op_count = r.outer_n;
        }
        return s;
    });
}

static int op_Ls(dwf_handle *h, int op_kind)
{
    return (op_kind == 1 && h->E->Ls_hat > 0) ? h->E->Ls : h->Ls;
}

dwf_status dwf_autotune(dwf_handle *h, dwf_prec prec, int op_kind)
{
    if (!h || !prec_ok(prec) || op_kind < 0 || op_kind > 1) return DWF_EINVAL;
    return guarded(&h->err, [&]() {
        h->E->autotune((Prec)prec, op_kind, op_Ls(h, op_kind));
        return DWF_OK;
    });
}

dwf_status dwf_get_kernel_config(dwf_handle *h, dwf_prec prec, int op_kind, dwf_kernel_config *c)
{
    if (!h || !c || !prec_ok(prec) || op_kind < 0 || op_kind > 1) return DWF_EINVAL;
    const Engine::KCfg &k = h->E->cfg[op_kind][prec];
    c->tile_sites = k.tile;
    c->gather = k.gather;
    return DWF_OK;
}

dwf_status dwf_set_kernel_config(dwf_handle *h, dwf_prec prec, int op_kind,
                                 const dwf_kernel_config *c)
{
    if (!h || !c || !prec_ok(prec) || op_kind < 0 || op_kind > 1) return DWF_EINVAL;
    if (c->tile_sites < 2 || c->tile_sites % 2 || c->gather < 0 || c->gather > 2) return DWF_EINVAL;
    const long seg = op_kind == 0 ? h->E->ne : (long)h->E->Nb_pad;
    if (seg % c->tile_sites || !stage_fits((Prec)prec, c->tile_sites, h->Ls, c->gather)) {
        h->err = "kernel configuration does not fit";
        return DWF_EINVAL;
    }
    Engine::KCfg &k = h->E->cfg[op_kind][prec];
    k.tile = c->tile_sites;
    k.gather = (prec == DWF_F64) ? 0 : c->gather;
    k.tuned = true;
    return DWF_OK;
}

dwf_status dwf_set_wait_policy(dwf_handle *h, long long max_polls, int force_timeout)
{
    if (!h) return DWF_EINVAL;
    if (max_polls > 0xFFFFFFFFll) return DWF_EINVAL;
    h->E->poll_limit = max_polls > 0 ? (unsigned)max_polls : 0u;
    h->E->force_timeout = force_timeout != 0;
    return DWF_OK;
}

const char *dwf_batch_last_error(const dwf_batch *bt) { return bt ? bt->err.c_str() : "null"; }

long long dwf_kernel_launch_count(void) { return launch_count(); }

}  // extern "C"
