// Device state of one or more lattices that are solved together: tables,
// fifth-dimension matrices, workspaces, operator composition and solvers.
#pragma once

#include <map>
#include <memory>
#include <string>
#include <vector>

#include "geometry.h"

namespace dwf {

// Two timing events, destroyed on every exit path.
struct EventPair {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    EventPair()
    {
        DWF_CUDA(cudaEventCreate(&e0));
        const cudaError_t e = cudaEventCreate(&e1);
        if (e != cudaSuccess) {
            cudaEventDestroy(e0);
            throw CudaError{e, "cudaEventCreate"};
        }
    }
    ~EventPair()
    {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    }
    EventPair(const EventPair &) = delete;
    EventPair &operator=(const EventPair &) = delete;
};

class Engine;

// Issues an engine's work on another stream for one scope: the engine's own
// stream comes back on every exit path, exceptions included.
struct StreamSwap {
    Engine &E;
    cudaStream_t old;
    StreamSwap(Engine &e, void *s);
    ~StreamSwap();
    StreamSwap(const StreamSwap &) = delete;
    StreamSwap &operator=(const StreamSwap &) = delete;
};

// Fifth-dimension matrices of one Ls for every system, [nsys][2][Ls][Ls]
// (chirality 0 = spins 0,1 (P_-), 1 = spins 2,3 (P_+)).
enum MatKind {
    MK_S1F = 0,  // M_phi M5^-1
    MK_M5I,      // M5^-1
    MK_M5ID,     // M5^-+
    MK_S3F,      // M5^-+ M_phi^+
    MK_S4F,      // M_phi^+
    MK_S4G,      // M5op^+
    MK_S2GF,     // M5^-+ M5^-1
    MK_MPHI,     // M_phi
    MK_N
};
// Operand A of the tensor-core products: [G | -F] (or F alone) in FP16,
// stored in the per-lane fragment order of mma m16n8k16:
// [nsys][chi][k-step 2][lane 32] x 8 halves.
enum TcKind {
    TC_S1 = 0,   // F = M_phi M5^-1
    TC_S2G,      // [M5^-+ | -M5^-+ M5^-1]
    TC_S2,       // [1 | -M5^-1]
    TC_S3,       // M5^-+ M_phi^+
    TC_S4,       // [M5op^+ | -M_phi^+]
    TC_M5I,      // M5^-1
    TC_M5ID,     // M5^-+
    TC_MPHI,     // M_phi
    TC_N
};
struct Mats {
    int Ls = 0;
    bool structured = false;  // |B / A| < 0.9: the recurrences of FProg are well damped
    double *d64[MK_N] = {};
    float *d32[MK_N] = {};
    void *tc[TC_N] = {};
    double *mphi = nullptr;  // [nsys][5] = (b, c, mass, A, B)
};

struct SysInfo {
    const LatticeGeom *g = nullptr;
    const double *gauge = nullptr;  // host, canonical
    double mass = 0;
    long off = 0;      // packed even offset of the system
    int blk_off = 0;   // first block of the system
};

class Engine {
  public:
    Engine() = default;
    ~Engine();
    Engine(const Engine &) = delete;

    // Build device tables for the given systems (same Ls, b, c, M5 and block
    // region shapes).
    void init(const std::vector<SysInfo> &sys, int Ls, double b, double c, double M5,
              cudaStream_t st);

    cudaStream_t st = 0;
    int Ls = 0;
    double b = 0, c = 0, M5 = 0;
    std::vector<SysInfo> sys;
    long ne = 0;               // packed even (= odd) sites, all systems
    int nblk = 0;              // blocks, all systems
    int Nb_pad = 0, O1_pad = 0, E2_pad = 0;
    long nO1 = 0, nE2 = 0;

    // device tables
    int *nbr_e = nullptr, *nbr_o = nullptr, *t1 = nullptr, *t2 = nullptr, *t3 = nullptr,
        *t4 = nullptr;
    // the local operator with Dirichlet walls on each hop (Eq. (eq:diri),
    // left side; an ablation of the snake terms), built on first use
    int *td1 = nullptr, *td2 = nullptr, *td3 = nullptr, *td4 = nullptr;
    bool local_truncated = false;
    void set_local_truncated(bool on);
    void local_tables(std::vector<int> *h, bool dirichlet) const;
    uint16_t *tsys_e = nullptr, *tsys_O1 = nullptr, *tsys_E2 = nullptr;  // null for 1 system
    Seg seg_sys, seg_blk;
    std::vector<long *> perm;  // per system: packed -> canonical cb (device)

    // links by precision class: 0 = FP64, 1 = FP32, 2 = half
    void *links(int which, Prec p);  // which: 0 even, 1 odd, 2 O1, 3 E2
    const Mats &mats(int Ls);

    // workspaces
    void *ws(const std::string &name, size_t bytes);
    // Blocks per preconditioner wave that keep the inner working set of a wave
    // within half of L2.
    int wave_blocks(Prec pi, int L);
    // page-locked host doubles (for asynchronous residual read-back)
    double *pinned_d(size_t n);
    cudaStream_t solve_stream = nullptr;  // private stream for graph-captured solves
    // Event pairs bracketing operator applications (time_kernels): slot 0 the
    // outer D^+D, slots 1.. the local operators of one preconditioner call.
    bool time_kernels = false;
    std::vector<cudaEvent_t> tev;  // 2 per slot
    std::vector<char> tev_used;
    void timed_begin(int slot);
    void timed_end(int slot);
    // mark slots whose events the stream has been asked to record (direct
    // launches or graph replays)
    void timed_mark(int first, int count);
    // sums elapsed times of the used slots (events must have completed)
    void timed_collect(double &outer_ms, long long &outer_n, double &local_ms, long long &local_n);
    // per-system activity during a batched solve (device; null outside solves)
    const int *active = nullptr;
    double *ws_d(const std::string &name, size_t n) { return (double *)ws(name, n * sizeof(double)); }

    // Operators on packed fields.  dot_part (optional): per-CTA partials of
    // <in, out> from the last stage; returns the CTA tile used.
    // scratch (optional): three caller-provided fields of field_bytes(p, ne, Ls)
    // bytes each, used instead of the engine's workspaces for t1, w, t3.
    // in_mphi (optional, D and D^+D): M_phi in, precomputed by the producer of
    // `in`; the first stage then gathers it without applying M_phi on load.
    int apply_global(Prec p, dwf_op op, void *out, const void *in, double *dot_part,
                     void *const *scratch = nullptr, const void *in_mphi = nullptr);
    // Has everything apply_global(p, ...) needs been created already (links,
    // matrices, launch configuration), so that it would allocate nothing?
    bool global_ready(Prec p) const;
    // blocks [b0, b1) only (b1 < 0: all); indices stay absolute
    int apply_local(Prec p, int Ls, void *out, const void *in, double *dot_part, int b0 = 0,
                    int b1 = -1, const void *in_mphi = nullptr);
    void apply_5d(Prec p, int Ls, MatKind k, void *out, const void *in, long nsite);

    // Launch configuration of the hop stages of one operator (0 = global
    // D^+D family, 1 = local operator) in one precision, chosen by autotune().
    struct KCfg {
        int tile = 8;
        int gather = 0;
        bool tuned = false;
    };
    KCfg cfg[2][kNumPrec];  // [global|local][Prec]
    bool autotune_on = true;
    // Times every fitting (tile, gather) candidate on this engine's lattice
    // and keeps the fastest; `which` 0 global, 1 local at fifth extent Ls_op.
    void autotune(Prec p, int which, int Ls_op, int reps = 5);
    const KCfg &kcfg(Prec p, int which, int Ls_op);
    // device flag raised by a bounded wait that gave up (reported as DWF_ETIMEOUT)
    int *err_flag = nullptr;
    // bounded-wait policy of the stage kernels (dwf_set_wait_policy)
    unsigned poll_limit = 0;
    int force_timeout = 0;
    // stage arguments common to every launch: error flag and wait policy
    StageArgs stage_base() const
    {
        StageArgs a{};
        a.err = err_flag;
        a.poll_limit = poll_limit;
        a.force_timeout = force_timeout;
        return a;
    }
    bool check_err();  // reads and clears the flag (synchronizes the stream)

    // reduced Ls
    int Ls_hat = 0;
    double mu = 0;
    float *Tm = nullptr;  // device (4 Ls_hat) x (4 Ls) complex

  private:
    void *lnk_[4][3] = {};
    std::map<int, Mats> mats_;
    std::map<std::string, std::pair<void *, size_t>> ws_;
    std::vector<void *> owned_;
    double *pinned_ = nullptr;
    size_t pinned_n_ = 0;
    template <class T> T *upload(const std::vector<T> &h);
};

inline StreamSwap::StreamSwap(Engine &e, void *s) : E(e), old(e.st)
{
    if (s) E.st = (cudaStream_t)s;
}
inline StreamSwap::~StreamSwap() { E.st = old; }

// Solver driver (solver.cu).  xs/bs: canonical FP64 device fields per system.
struct SolveResult {
    int iters = 0, inner_total = 0, ru = 0, converged = 0;
    std::vector<double> true_res;
    double ms = 0;
    long long launches = 0;
    double local_ms = 0, outer_ms = 0;  // with time_kernels
    long long local_n = 0, outer_n = 0;
};
dwf_status solve(Engine &E, double *const *xs, const double *const *bs, const dwf_solver_params &p,
                 bool precond, SolveResult &res, std::string &err);
// z = M^-1 r for FP64 canonical fields (single system)
void precondition_fp64(Engine &E, double *z, const double *r, const dwf_solver_params &p);
void reduced_local_inverse(Engine &E, double *out, const double *in, int Ls_hat, int iters,
                           const dwf_solver_params &P);

}  // namespace dwf
