// Engine: device tables, fifth-dimension matrices and operator composition.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <stdexcept>

#include <cuda_fp16.h>

#include "engine.h"

namespace dwf {

// Local stage tables of all systems, concatenated with block offsets.  With
// dirichlet, only hops between sites inside the block are kept: the four hops
// of D^+D then each see Dirichlet walls at the block boundary, the left side
// of Eq. (eq:diri) (the snake terms dropped; outputs outside the block are 0).
void Engine::local_tables(std::vector<int> *h, bool dirichlet) const
{
    const int Nb = sys[0].g->Nb;  // every system has the same block shape
    auto inside = [](int e, int pad, int nb) {
        const long idx = e >= 0 ? (long)e : (long)(-e - 2);
        return idx % pad < nb;
    };
    auto add = [&](std::vector<int> &dst, const std::vector<int> &src, long off, int out_pad, int in_pad) {
        const long rows = (long)src.size() / 8;
        for (long r = 0; r < rows; r++) {
            const bool out_in = (r % out_pad) < Nb;
            for (int k = 0; k < 8; k++) {
                const int e = src[r * 8 + k];
                if (e == -1 || (dirichlet && (!out_in || !inside(e, in_pad, Nb)))) {
                    dst.push_back(-1);
                } else if (e >= 0) {
                    dst.push_back((int)(e + off));
                } else {
                    dst.push_back((int)(-(((long)-e - 2) + off) - 2));
                }
            }
        }
    };
    for (int k = 0; k < 4; k++) h[k].clear();
    for (auto &sy : sys) {
        const LatticeGeom &g = *sy.g;
        const long bo = sy.blk_off;
        add(h[0], g.t1, bo * Nb_pad, O1_pad, Nb_pad);  // O1 <- interior
        add(h[1], g.t2, bo * O1_pad, E2_pad, O1_pad);  // E2 <- O1
        add(h[2], g.t3, bo * E2_pad, O1_pad, E2_pad);  // O1 <- E2
        add(h[3], g.t4, bo * O1_pad, Nb_pad, O1_pad);  // interior <- O1
    }
}

void Engine::set_local_truncated(bool on)
{
    if (on && !td1) {
        std::vector<int> h[4];
        local_tables(h, true);
        td1 = upload(h[0]);
        td2 = upload(h[1]);
        td3 = upload(h[2]);
        td4 = upload(h[3]);
    }
    local_truncated = on;
}

// Under stream capture the record must be an external event node, so that
// every replay of the graph re-records the event; outside capture the flag is
// refused and a plain record is taken.
static void record_timing_event(cudaEvent_t ev, cudaStream_t st)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    DWF_CUDA(cudaStreamIsCapturing(st, &cs));
    if (cs == cudaStreamCaptureStatusActive)
        DWF_CUDA(cudaEventRecordWithFlags(ev, st, cudaEventRecordExternal));
    else
        DWF_CUDA(cudaEventRecord(ev, st));
}

void Engine::timed_begin(int slot)
{
    if (!time_kernels) return;
    if ((int)tev_used.size() <= slot) {
        const int old = (int)tev_used.size();
        tev.resize(2 * (slot + 1));
        tev_used.resize(slot + 1, 0);
        for (int k = 2 * old; k < 2 * (slot + 1); k++) DWF_CUDA(cudaEventCreate(&tev[k]));
    }
    record_timing_event(tev[2 * slot], st);
}

void Engine::timed_end(int slot)
{
    if (!time_kernels) return;
    record_timing_event(tev[2 * slot + 1], st);
}

void Engine::timed_mark(int first, int count)
{
    if (!time_kernels) return;
    for (int k = first; k < first + count && k < (int)tev_used.size(); k++) tev_used[k] = 1;
}

void Engine::timed_collect(double &outer_ms, long long &outer_n, double &local_ms, long long &local_n)
{
    for (size_t k = 0; k < tev_used.size(); k++) {
        if (!tev_used[k]) continue;
        float ms = 0;
        if (cudaEventElapsedTime(&ms, tev[2 * k], tev[2 * k + 1]) != cudaSuccess) {
            cudaGetLastError();  // timing unavailable for this pair: skip it
            tev_used[k] = 0;
            continue;
        }
        if (k == 0) {
            outer_ms += ms;
            outer_n++;
        } else {
            local_ms += ms;
            local_n++;
        }
        tev_used[k] = 0;
    }
}

Engine::~Engine()
{
    for (cudaEvent_t ev : tev) cudaEventDestroy(ev);
    for (void *p : owned_) cudaFree(p);
    for (auto &kv : ws_) cudaFree(kv.second.first);
    if (pinned_) cudaFreeHost(pinned_);
    if (solve_stream) cudaStreamDestroy(solve_stream);
}

double *Engine::pinned_d(size_t n)
{
    if (pinned_n_ < n) {
        if (pinned_) {
            DWF_CUDA(cudaStreamSynchronize(st));
            cudaFreeHost(pinned_);
            pinned_ = nullptr;
        }
        DWF_CUDA(cudaMallocHost(&pinned_, n * sizeof(double)));
        pinned_n_ = n;
    }
    return pinned_;
}

template <class T>
T *Engine::upload(const std::vector<T> &h)
{
    if (h.empty()) return nullptr;
    T *d = nullptr;
    DWF_CUDA(cudaMalloc(&d, h.size() * sizeof(T)));
    owned_.push_back(d);
    DWF_CUDA(cudaMemcpy(d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
    return d;
}

void *Engine::ws(const std::string &name, size_t bytes)
{
    auto it = ws_.find(name);
    if (it != ws_.end() && it->second.second >= bytes) return it->second.first;
    if (it != ws_.end()) {
        DWF_CUDA(cudaStreamSynchronize(st));
        cudaFree(it->second.first);
        ws_.erase(it);
    }
    void *p = nullptr;
    DWF_CUDA(cudaMalloc(&p, std::max<size_t>(bytes, 256)));
    DWF_CUDA(cudaMemsetAsync(p, 0, std::max<size_t>(bytes, 256), st));
    ws_[name] = {p, bytes};
    return p;
}

void Engine::init(const std::vector<SysInfo> &sysv, int Ls_, double b_, double c_, double M5_,
                  cudaStream_t st_)
{
    sys = sysv;
    Ls = Ls_;
    b = b_;
    c = c_;
    M5 = M5_;
    st = st_;
    const LatticeGeom &g0 = *sys[0].g;
    Nb_pad = g0.Nb_pad;
    O1_pad = g0.O1_pad;
    E2_pad = g0.E2_pad;
    ne = 0;
    nblk = 0;
    for (auto &s : sys) {
        if (s.g->Nb_pad != Nb_pad || s.g->O1_pad != O1_pad || s.g->E2_pad != E2_pad)
            throw std::runtime_error("systems of a batch need identical block regions");
        s.off = ne;
        s.blk_off = nblk;
        ne += s.g->ne();
        nblk += s.g->nblk;
    }
    nO1 = (long)nblk * O1_pad;
    nE2 = (long)nblk * E2_pad;

    // concatenated tables with offsets
    auto shift = [](std::vector<int> &dst, const std::vector<int> &src, long off) {
        for (int e : src) {
            if (e == -1) dst.push_back(-1);
            else if (e >= 0) dst.push_back((int)(e + off));
            else dst.push_back((int)(-(((long)-e - 2) + off) - 2));
        }
    };
    std::vector<int> he, ho;
    for (auto &s : sys) {
        shift(he, s.g->nbr_e, s.off);
        shift(ho, s.g->nbr_o, s.off);
    }
    nbr_e = upload(he);
    nbr_o = upload(ho);
    {
        std::vector<int> h[4];
        local_tables(h, false);
        t1 = upload(h[0]);
        t2 = upload(h[1]);
        t3 = upload(h[2]);
        t4 = upload(h[3]);
    }

    // per-tile system ids (only needed for several systems)
    if (sys.size() > 1) {
        std::vector<uint16_t> te, tO1, tE2;
        for (size_t k = 0; k < sys.size(); k++) {
            te.insert(te.end(), sys[k].g->ne() / kSegPad, (uint16_t)k);
            tO1.insert(tO1.end(), (long)sys[k].g->nblk * O1_pad / kSegPad, (uint16_t)k);
            tE2.insert(tE2.end(), (long)sys[k].g->nblk * E2_pad / kSegPad, (uint16_t)k);
        }
        tsys_e = upload(te);
        tsys_O1 = upload(tO1);
        tsys_E2 = upload(tE2);
    }
    // segments: systems and blocks over the packed even space
    {
        std::vector<uint16_t> ts;
        seg_sys.nseg = (int)sys.size();
        seg_sys.h_tile_begin.clear();
        for (size_t k = 0; k < sys.size(); k++) {
            seg_sys.h_tile_begin.push_back((int)(sys[k].off / kSegPad));
            ts.insert(ts.end(), sys[k].g->ne() / kSegPad, (uint16_t)k);
        }
        seg_sys.h_tile_begin.push_back((int)(ne / kSegPad));
        seg_sys.d_tile_seg = upload(ts);
        seg_sys.d_tile_begin = upload(seg_sys.h_tile_begin);
        seg_sys.nsite = ne;
    }
    {
        if (nblk > 65535) throw std::runtime_error("too many blocks");
        std::vector<uint16_t> ts;
        seg_blk.nseg = nblk;
        seg_blk.h_tile_begin.clear();
        const int tpb = Nb_pad / kSegPad;
        for (int k = 0; k < nblk; k++) {
            seg_blk.h_tile_begin.push_back(k * tpb);
            ts.insert(ts.end(), tpb, (uint16_t)k);
        }
        seg_blk.h_tile_begin.push_back(nblk * tpb);
        seg_blk.d_tile_seg = upload(ts);
        seg_blk.d_tile_begin = upload(seg_blk.h_tile_begin);
        seg_blk.nsite = ne;
    }
    perm.clear();
    for (auto &s : sys) perm.push_back(upload(s.g->even_cb));
    err_flag = upload(std::vector<int>(1, 0));
}

int Engine::wave_blocks(Prec pi, int L)
{
    int dev = 0, l2 = 0;
    DWF_CUDA(cudaGetDevice(&dev));
    DWF_CUDA(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev));
    const size_t vec = 3 * field_bytes(pi, Nb_pad, L) + field_bytes(P32, Nb_pad, L);
    const size_t halo = field_bytes(pi, 2L * O1_pad + E2_pad, L);
    const size_t lnk = (size_t)(O1_pad + E2_pad) * 8 * 12 * 2;
    const size_t tab = (size_t)(2L * O1_pad + E2_pad + Nb_pad) * 8 * 4;
    const size_t per_block = vec + halo + lnk + tab;
    const long w = (long)(0.5 * l2) / (long)per_block;
    return (int)std::max<long>(1, std::min<long>(w, nblk));
}

bool Engine::check_err()
{
    int h = 0;
    DWF_CUDA(cudaMemcpyAsync(&h, err_flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    DWF_CUDA(cudaStreamSynchronize(st));
    if (h) DWF_CUDA(cudaMemsetAsync(err_flag, 0, sizeof(int), st));
    return h != 0;
}

void *Engine::links(int which, Prec p)
{
    const int cls = p == P64 ? 0 : p == P32 ? 1 : 2;
    if (lnk_[which][cls]) return lnk_[which][cls];
    std::vector<unsigned char> all, part;
    for (auto &s : sys) {
        const LatticeGeom &g = *s.g;
        const std::vector<long> &src = which == 0 ? g.lnk_e : which == 1 ? g.lnk_o : which == 2 ? g.lnk_O1 : g.lnk_E2;
        gather_links(src, s.gauge, cls == 0 ? P64 : cls == 1 ? P32 : P16, part);
        all.insert(all.end(), part.begin(), part.end());
    }
    lnk_[which][cls] = upload(all);
    return lnk_[which][cls];
}

// ------------------------------------------------------------ 5D matrices
namespace {
using Mat = std::vector<double>;  // Ls x Ls row-major

Mat matmul(const Mat &a, const Mat &b, int n)
{
    Mat c(n * n, 0.0);
    for (int i = 0; i < n; i++)
        for (int k = 0; k < n; k++)
            for (int j = 0; j < n; j++) c[i * n + j] += a[i * n + k] * b[k * n + j];
    return c;
}
Mat transpose(const Mat &a, int n)
{
    Mat t(n * n);
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) t[j * n + i] = a[i * n + j];
    return t;
}
Mat inverse(Mat a, int n)
{
    Mat inv(n * n, 0.0);
    for (int i = 0; i < n; i++) inv[i * n + i] = 1.0;
    for (int col = 0; col < n; col++) {
        int piv = col;
        for (int r = col + 1; r < n; r++)
            if (std::fabs(a[r * n + col]) > std::fabs(a[piv * n + col])) piv = r;
        for (int j = 0; j < n; j++) {
            std::swap(a[col * n + j], a[piv * n + j]);
            std::swap(inv[col * n + j], inv[piv * n + j]);
        }
        const double d = a[col * n + col];
        for (int j = 0; j < n; j++) {
            a[col * n + j] /= d;
            inv[col * n + j] /= d;
        }
        for (int r = 0; r < n; r++) {
            if (r == col) continue;
            const double f = a[r * n + col];
            if (f == 0.0) continue;
            for (int j = 0; j < n; j++) {
                a[r * n + j] -= f * a[col * n + j];
                inv[r * n + j] -= f * inv[col * n + j];
            }
        }
    }
    return inv;
}
}  // namespace

const Mats &Engine::mats(int L)
{
    auto it = mats_.find(L);
    if (it != mats_.end()) return it->second;
    Mats m;
    m.Ls = L;
    const size_t per = 2 * (size_t)L * L;
    std::vector<double> h[MK_N];
    for (auto &hk : h) hk.assign(per * sys.size(), 0.0);
    std::vector<double> mp;
    const double A = b * (4.0 - M5) + 1.0, B = c * (4.0 - M5) - 1.0;
    m.structured = A != 0.0 && std::fabs(B / A) < 0.9;
    for (size_t k = 0; k < sys.size(); k++) {
        const double mass = sys[k].mass;
        mp.push_back(b);
        mp.push_back(c);
        mp.push_back(mass);
        mp.push_back(A);
        mp.push_back(B);
        for (int chi = 0; chi < 2; chi++) {
            // chirality 0 (spins 0,1): (P psi)_s = psi_{s+1}; 1 (spins 2,3): psi_{s-1}; wraps -mass
            Mat P(L * L, 0.0), I(L * L, 0.0);
            for (int s = 0; s < L; s++) {
                I[s * L + s] = 1.0;
                if (chi == 0) {
                    if (s + 1 < L) P[s * L + s + 1] += 1.0;
                    else P[s * L + 0] += -mass;
                } else {
                    if (s >= 1) P[s * L + s - 1] += 1.0;
                    else P[0 * L + L - 1] += -mass;
                }
            }
            Mat M5op(L * L), Mphi(L * L);
            for (int e = 0; e < L * L; e++) {
                M5op[e] = A * I[e] + B * P[e];
                Mphi[e] = -0.5 * (b * I[e] + c * P[e]);
            }
            const Mat M5i = inverse(M5op, L);
            const Mat M5iT = transpose(M5i, L), MphiT = transpose(Mphi, L), M5opT = transpose(M5op, L);
            const Mat out[MK_N] = {matmul(Mphi, M5i, L), M5i, M5iT, matmul(M5iT, MphiT, L), MphiT,
                                   M5opT, matmul(M5iT, M5i, L), Mphi};
            for (int q = 0; q < MK_N; q++)
                std::copy(out[q].begin(), out[q].end(), h[q].begin() + k * per + chi * (size_t)L * L);
        }
    }
    for (int q = 0; q < MK_N; q++) {
        m.d64[q] = upload(h[q]);
        std::vector<float> f(h[q].begin(), h[q].end());
        m.d32[q] = upload(f);
    }
    // tensor-core operand A per kind: k-step 0 and 1 matrices (null = zero)
    if (L <= 16) {
        const size_t nsys = sys.size();
        std::vector<double> ident(per * nsys, 0.0), neg[MK_N];
        for (size_t k = 0; k < nsys; k++)
            for (int chi = 0; chi < 2; chi++)
                for (int s = 0; s < L; s++) ident[k * per + chi * L * L + s * L + s] = 1.0;
        for (int q = 0; q < MK_N; q++) {
            neg[q] = h[q];
            for (double &v : neg[q]) v = -v;
        }
        const std::vector<double> *src[TC_N][2] = {
            {&h[MK_S1F], nullptr},  {&h[MK_M5ID], &neg[MK_S2GF]}, {&ident, &neg[MK_M5I]},
            {&h[MK_S3F], nullptr},  {&h[MK_S4G], &neg[MK_S4F]},   {&h[MK_M5I], nullptr},
            {&h[MK_M5ID], nullptr}, {&h[MK_MPHI], nullptr}};
        for (int q = 0; q < TC_N; q++) {
            std::vector<__half> frag(nsys * 2 * 2 * 32 * 8, __float2half(0.f));
            for (size_t k = 0; k < nsys; k++)
                for (int chi = 0; chi < 2; chi++)
                    for (int kk = 0; kk < 2; kk++) {
                        const std::vector<double> *M = src[q][kk];
                        if (!M) continue;
                        auto A = [&](int r, int c) -> double {
                            return (r < L && c < L) ? (*M)[k * per + chi * L * L + r * L + c] : 0.0;
                        };
                        for (int lane = 0; lane < 32; lane++) {
                            const int g = lane >> 2, tg = lane & 3;
                            const double v[8] = {A(g, 2 * tg),     A(g, 2 * tg + 1),
                                                 A(g + 8, 2 * tg), A(g + 8, 2 * tg + 1),
                                                 A(g, 2 * tg + 8), A(g, 2 * tg + 9),
                                                 A(g + 8, 2 * tg + 8), A(g + 8, 2 * tg + 9)};
                            __half *dst = frag.data() + ((((k * 2 + chi) * 2 + kk) * 32 + lane) * 8);
                            for (int e = 0; e < 8; e++) dst[e] = __float2half_rn((float)v[e]);
                        }
                    }
            m.tc[q] = upload(frag);
        }
    }
    m.mphi = upload(mp);
    return mats_[L] = m;
}

// ------------------------------------------------------------ operators
static const void *matp(const Mats &m, MatKind k, Prec p)
{
    return p == P64 ? (const void *)m.d64[k] : (const void *)m.d32[k];
}

static bool is_half(Prec p) { return p == P16 || p == PB16 || p == PFX16 || p == PFX8; }

// Matrices of a stage: CUDA-core path F (and G), tensor-core path the fused
// operand A; G is kept non-null on the tensor-core path only as a flag.
static void set_mats(StageArgs &a, const Mats &m, Prec p, MatKind f, MatKind g, TcKind tc)
{
    if (is_half(p)) {
        if (!m.tc[tc]) throw std::runtime_error("tensor-core path needs Ls <= 16");
        a.F = m.tc[tc];
        a.G = (g == MK_N) ? nullptr : m.tc[tc];
    } else {
        a.F = matp(m, f, p);
        a.G = (g == MK_N) ? nullptr : matp(m, g, p);
        a.fprog = FP_DENSE;
        // structured where it beats the dense product (measured: S2's two
        // products; a single F product in S1 / S3 is as fast dense)
        if (m.structured && m.Ls <= 32) {
            if (f == MK_M5I && g == MK_N) a.fprog = FP_M5I;
            else if (f == MK_M5ID && g == MK_N) a.fprog = FP_M5ID;
            else if (f == MK_S2GF && g == MK_M5ID) a.fprog = FP_S2;
        }
    }
}

void Engine::apply_5d(Prec p, int L, MatKind k, void *out, const void *in, long nsite)
{
    const Mats &m = mats(L);
    StageArgs a = stage_base();
    a.in = in;
    a.out = out;
    a.mphi = m.mphi;
    set_mats(a, m, p, k, MK_N, k == MK_M5I ? TC_M5I : k == MK_M5ID ? TC_M5ID : TC_MPHI);
    a.tile_sys = (nsite == ne) ? tsys_e : nullptr;
    a.nout = nsite;
    a.nin = nsite;
    a.Ls = L;
    a.tile = 8;
    a.seg_out = (int)std::min<long>(nsite, 1 << 30);
    a.link_stride = a.seg_out;
    launch_stage(p, MODE_5D, false, a, st);
}

const Engine::KCfg &Engine::kcfg(Prec p, int which, int Ls_op)
{
    KCfg &c = cfg[which][p];
    if (!c.tuned && autotune_on) autotune(p, which, Ls_op);
    return c;
}

void Engine::autotune(Prec p, int which, int Ls_op, int reps)
{
    KCfg &c = cfg[which][p];
    c.tuned = true;  // also guards the recursion through apply_*
    c.tile = 8;
    c.gather = 0;
    const long n = ne;
    void *x = ws("tune_x", field_bytes(p, n, Ls_op));
    void *y = ws("tune_y", field_bytes(p, n, Ls_op));
    // finite, normal values in every storage format (and in the FP16 scales)
    DWF_CUDA(cudaMemsetAsync(x, 0x3c, field_bytes(p, n, Ls_op), st));
    EventPair ev;
    std::vector<KCfg> cand;
    const int tiles[] = {4, 8, 16, 32};
    const int ngather = (p == P64 || p == PFX8) ? 1 : (p == P32 ? 2 : 3);
    for (int gather = 0; gather < ngather; gather++)
        for (int tile : tiles) {
            if (!stage_fits(p, tile, Ls_op, gather)) continue;
            if ((which == 0 ? ne : (long)Nb_pad) % tile) continue;
            KCfg k = c;
            k.tile = tile;
            k.gather = gather;
            cand.push_back(k);
        }
    // two rounds over the candidates, each kept at its faster round (one
    // noisy measurement must not decide)
    std::vector<float> tbest(cand.size(), 1e30f);
    try {
        for (int round = 0; round < 2; round++)
            for (size_t q = 0; q < cand.size(); q++) {
                c.tile = cand[q].tile;
                c.gather = cand[q].gather;
                // timed on the solvers' path, whose first stage reads M_phi x
                // written beforehand (x stands in for it here)
                auto run = [&]() {
                    if (which == 0) apply_global(p, DWF_OP_DDAGD, y, x, nullptr, nullptr, x);
                    else apply_local(p, Ls_op, y, x, nullptr, 0, -1, x);
                };
                run();
                DWF_CUDA(cudaEventRecord(ev.e0, st));
                for (int r = 0; r < reps; r++) run();
                DWF_CUDA(cudaEventRecord(ev.e1, st));
                DWF_CUDA(cudaEventSynchronize(ev.e1));
                float ms = 0;
                DWF_CUDA(cudaEventElapsedTime(&ms, ev.e0, ev.e1));
                tbest[q] = std::min(tbest[q], ms);
            }
    } catch (...) {
        // a failed tuning run leaves the default shape, not the candidate it was timing
        c.tile = 8;
        c.gather = 0;
        throw;
    }
    KCfg bestc = c;
    float best = 1e30f;
    for (size_t q = 0; q < cand.size(); q++)
        if (tbest[q] < best) {
            best = tbest[q];
            bestc = cand[q];
        }
    c = bestc;
    c.tuned = true;
}

bool Engine::global_ready(Prec p) const
{
    const int cls = p == P64 ? 0 : p == P32 ? 1 : 2;
    return lnk_[0][cls] && lnk_[1][cls] && mats_.count(Ls) && cfg[0][p].tuned;
}

int Engine::apply_global(Prec p, dwf_op op, void *out, const void *in, double *dot_part,
                         void *const *scratch, const void *in_mphi)
{
    const Mats &m = mats(Ls);
    const size_t fb = field_bytes(p, ne, Ls);
    const std::string tag = std::to_string((int)p);
    void *t1v = scratch ? scratch[0] : ws("g_t1_" + tag, fb);
    void *wv = scratch ? scratch[1] : ws("g_w_" + tag, fb);
    void *t3v = scratch ? scratch[2] : ws("g_t3_" + tag, fb);
    const KCfg kc = kcfg(p, 0, Ls);
    const int tile = kc.tile;
    if (kc.gather == 2 && !in_mphi && (op == DWF_OP_D || op == DWF_OP_DDAGD)) {
        // the tensor-core hop reads M_phi x precomputed: write it into the w
        // field, which the first stage reads and the second overwrites
        apply_5d(p, Ls, MK_MPHI, wv, in, ne);
        in_mphi = wv;
    }

    StageArgs base = stage_base();
    base.gather = kc.gather;
    base.active = active;
    base.tile_sys = tsys_e;
    base.mphi = m.mphi;
    base.nout = ne;
    base.nin = ne;
    base.naux = ne;
    base.Ls = Ls;
    base.tile = tile;
    base.seg_out = (int)ne;
    base.link_stride = (int)ne;
    base.aux_stride = (int)ne;
    base.aux_valid = (int)ne;

    auto S1 = [&](const void *x) {
        StageArgs a = base;
        a.in = in_mphi ? in_mphi : x;
        a.out = t1v;
        a.nbr = nbr_o;
        a.links = links(1, p);
        set_mats(a, m, p, MK_S1F, MK_N, TC_S1);
        launch_stage(p, MODE_F, in_mphi == nullptr, a, st);
    };
    auto S2 = [&](const void *x, void *o, bool with_g) {
        StageArgs a = base;
        a.in = t1v;
        a.out = o;
        a.nbr = nbr_e;
        a.links = links(0, p);
        a.aux = x;
        if (with_g) set_mats(a, m, p, MK_S2GF, MK_M5ID, TC_S2G);
        else set_mats(a, m, p, MK_M5I, MK_N, TC_S2);
        launch_stage(p, MODE_S2, false, a, st);
    };
    auto S3 = [&](const void *w) {
        StageArgs a = base;
        a.in = w;
        a.out = t3v;
        a.nbr = nbr_o;
        a.links = links(1, p);
        set_mats(a, m, p, MK_S3F, MK_N, TC_S3);
        a.dagger = 1;
        launch_stage(p, MODE_F, false, a, st);
    };
    auto S4 = [&](const void *w, void *o, const void *dotv) {
        StageArgs a = base;
        a.in = t3v;
        a.out = o;
        a.nbr = nbr_e;
        a.links = links(0, p);
        a.aux = w;
        set_mats(a, m, p, MK_S4F, MK_S4G, TC_S4);
        a.dagger = 1;
        a.dotv = dotv;
        a.dot_part = dot_part;
        launch_stage(p, MODE_S4, false, a, st);
    };
    switch (op) {
    case DWF_OP_D:
        S1(in);
        S2(in, out, false);
        break;
    case DWF_OP_DDAG:
        apply_5d(p, Ls, MK_M5ID, wv, in, ne);
        S3(wv);
        S4(wv, out, in);
        break;
    case DWF_OP_DDAGD:
        S1(in);
        S2(in, wv, true);
        S3(wv);
        S4(wv, out, in);
        break;
    default: throw std::runtime_error("apply_global: bad op");
    }
    return tile;
}

int Engine::apply_local(Prec p, int L, void *out, const void *in, double *dot_part, int b0, int b1,
                        const void *in_mphi)
{
    if (b1 < 0) b1 = nblk;
    const Mats &m = mats(L);
    const std::string tag = std::to_string((int)p) + "_" + std::to_string(L);
    void *t1v = ws("l_t1_" + tag, field_bytes(p, nO1, L));
    void *wv = ws("l_w_" + tag, field_bytes(p, nE2, L));
    void *t3v = ws("l_t3_" + tag, field_bytes(p, nO1, L));
    const KCfg kc = kcfg(p, 1, L);
    const int tile = kc.tile;
    const long nI = (long)nblk * Nb_pad;
    if (kc.gather == 2 && !in_mphi) {
        // the tensor-core hop reads M_phi x precomputed
        void *u = ws("l_u_" + tag, field_bytes(p, nI, L));
        apply_5d(p, L, MK_MPHI, u, in, nI);
        in_mphi = u;
    }

    StageArgs a = stage_base();
    a.gather = kc.gather;
    a.active = active;
    a.mphi = m.mphi;
    a.Ls = L;
    a.tile = tile;
    // S1: O1 <- interior (M_phi applied on load unless the producer gave in_mphi)
    a.in = in_mphi ? in_mphi : in;
    a.nin = nI;
    a.out = t1v;
    a.nout = nO1;
    a.nbr = local_truncated ? td1 : t1;
    a.links = links(2, p);
    a.tile_sys = tsys_O1;
    a.seg_out = O1_pad;
    a.link_stride = O1_pad;
    a.site0 = (long)b0 * O1_pad;
    a.site_end = (long)b1 * O1_pad;
    set_mats(a, m, p, MK_S1F, MK_N, TC_S1);
    launch_stage(p, MODE_F, in_mphi == nullptr, a, st);
    // S2: E2 <- O1, aux = interior x
    StageArgs b2 = stage_base();
    b2.gather = kc.gather;
    b2.active = active;
    b2.mphi = m.mphi;
    b2.Ls = L;
    b2.tile = tile;
    b2.in = t1v;
    b2.nin = nO1;
    b2.out = wv;
    b2.nout = nE2;
    b2.nbr = local_truncated ? td2 : t2;
    b2.links = links(3, p);
    b2.tile_sys = tsys_E2;
    b2.seg_out = E2_pad;
    b2.link_stride = E2_pad;
    b2.site0 = (long)b0 * E2_pad;
    b2.site_end = (long)b1 * E2_pad;
    b2.aux = in;
    b2.naux = nI;
    b2.aux_stride = Nb_pad;
    b2.aux_valid = Nb_pad;
    set_mats(b2, m, p, MK_S2GF, MK_M5ID, TC_S2G);
    launch_stage(p, MODE_S2, false, b2, st);
    // S3: O1 <- E2 (dagger)
    StageArgs b3 = stage_base();
    b3.gather = kc.gather;
    b3.active = active;
    b3.mphi = m.mphi;
    b3.Ls = L;
    b3.tile = tile;
    b3.in = wv;
    b3.nin = nE2;
    b3.out = t3v;
    b3.nout = nO1;
    b3.nbr = local_truncated ? td3 : t3;
    b3.links = links(2, p);
    b3.tile_sys = tsys_O1;
    b3.seg_out = O1_pad;
    b3.link_stride = O1_pad;
    b3.site0 = (long)b0 * O1_pad;
    b3.site_end = (long)b1 * O1_pad;
    set_mats(b3, m, p, MK_S3F, MK_N, TC_S3);
    b3.dagger = 1;
    launch_stage(p, MODE_F, false, b3, st);
    // S4: interior <- O1 (dagger), aux = w
    StageArgs b4 = stage_base();
    b4.gather = kc.gather;
    b4.active = active;
    b4.Ls = L;
    b4.tile = tile;
    b4.in = t3v;
    b4.nin = nO1;
    b4.out = out;
    b4.nout = nI;
    b4.nbr = local_truncated ? td4 : t4;
    b4.links = links(3, p);
    b4.tile_sys = tsys_e;
    b4.seg_out = Nb_pad;
    b4.link_stride = E2_pad;
    b4.site0 = (long)b0 * Nb_pad;
    b4.site_end = (long)b1 * Nb_pad;
    b4.aux = wv;
    b4.naux = nE2;
    b4.aux_stride = E2_pad;
    b4.aux_valid = Nb_pad;
    set_mats(b4, m, p, MK_S4F, MK_S4G, TC_S4);
    b4.dagger = 1;
    b4.mphi = m.mphi;
    b4.dotv = in;
    b4.dot_part = dot_part;
    launch_stage(p, MODE_S4, false, b4, st);
    return tile;
}

}  // namespace dwf
