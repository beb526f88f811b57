/*
 * dwf.h -- C ABI of the GB300 (sm_103a) Mobius domain-wall solver library.
 *
 * The library solves the even-odd preconditioned Mobius domain-wall normal
 * equations D^+D psi_e = b (arXiv:2104.05615, Sec. 2.2, Eq. (normal_equation))
 * with plain CG or with the multi-splitting preconditioned CG (MSPCG,
 * Sec. 2.4, Algorithm 1) whose preconditioner runs a fixed number of inner
 * CG iterations (Sec. 2.5) on the local normal operator of every subdomain
 * block, snake terms included (Sec. 2.3), optionally through the reduced-Ls
 * transform of Sec. 3.3.
 *
 * Conventions
 *   - Lattice sites: lex = x + Lx*(y + Ly*(z + Lz*t)); parity (x+y+z+t) % 2
 *     (Sec. 2.2).  All four extents and all block extents must be even.
 *   - Canonical even/odd 5D field (the ABI vector layout): element
 *     ((s*(V/2) + lex/2)*4 + spin)*3 + colour, complex interleaved (re, im),
 *     over the sites of one parity.  Element type by precision:
 *       DWF_F64: double[2], DWF_F32: float[2], DWF_F16: IEEE half[2],
 *       DWF_BF16: bfloat16[2], DWF_FX16 and DWF_FX8: float[2] (the fixed-point
 *       formats are device storage formats only; they are exchanged as FP32).
 *   - Gauge field (host, FP64): ((lex*4 + mu)*3 + row)*3 + col complex
 *     (double[2]); mu = x, y, z, t; links must be SU(3) to ~1e-14 (the device
 *     copies keep two rows and rebuild the third).
 *   - Gamma basis: chiral (DeGrand-Rossi), gamma5 = diag(-1,-1,+1,+1).
 *   - Fifth dimension: M5op = A + B P, M_phi = -(b + c P)/2 with
 *     A = b(4-M5)+1, B = c(4-M5)-1, (P psi)_s = P_- psi_{s+1} + P_+ psi_{s-1}
 *     and -mass on the wrap terms (Mobius form, cited in Sec. 2.2).
 *   - Pointers named *_dev are device memory owned by the caller (e.g. a
 *     torch tensor); *_host are host memory owned by the caller.  The handle
 *     owns its copies of the gauge field, its tables and its workspaces.
 *   - Every call returns a dwf_status; nothing is thrown and no device trap
 *     is ever raised.  dwf_last_error() gives a one-line description.
 *   - Calls on one handle must not overlap (the handle's workspaces are
 *     shared).  Work is issued on the handle's stream (dwf_create); entry
 *     points that take a stream argument use that stream instead.
 */
#ifndef DWF_H
#define DWF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dwf_handle dwf_handle;
typedef struct dwf_batch dwf_batch;

typedef enum {
    DWF_OK = 0,
    DWF_EINVAL = 1,        /* bad argument (dims, block dims, null pointer, precision) */
    DWF_ENOMEM = 2,        /* device or host allocation failed */
    DWF_ECUDA = 3,         /* a CUDA runtime call failed */
    DWF_ENOCONV = 4,       /* solver reached maxiter; x holds the last iterate */
    DWF_ETIMEOUT = 5,      /* a bounded device-side wait gave up */
    DWF_EUNSUPPORTED = 6   /* valid but not implemented combination */
} dwf_status;

/* DWF_FX16: the 16-bit fixed-point format of Sec. 3.2 (Eq. for the fixed-point
 * value): every colour-spinor (24 reals at one site and s) is stored as 24
 * int16 integers q with one FP32 number, value = q / 32767 * max|component|
 * (the FP32 number kept is max/32767); loads unpack to FP32 and all
 * arithmetic is FP32, the fifth-dimension products on the tensor cores. */
/* DWF_FX8: the 8-bit fixed-point format of the same section: 24 int8 integers
 * per colour-spinor with one FP32 number, value = q / 127 * max|component|
 * (the FP32 number kept is max/127), stored as three 8-byte chunks per 5D site.
 * Like DWF_FX16 it is exchanged as FP32 and computed in FP32; its stages load
 * neighbours directly (gather 0 only). */
typedef enum { DWF_F64 = 0, DWF_F32 = 1, DWF_F16 = 2, DWF_BF16 = 3, DWF_FX16 = 4, DWF_FX8 = 5 } dwf_prec;

typedef enum {
    DWF_OP_D = 0,           /* D = 1 - M5^-1 M4_eo M5^-1 M4_oe (Sec. 2.2, Eq. dirac_equation) */
    DWF_OP_DDAG = 1,        /* D^+ */
    DWF_OP_DDAGD = 2,       /* D^+D (Sec. 2.2, Eq. normal_equation) */
    DWF_OP_LOCAL_DDAGD = 3, /* (+)_s R_s D^+D R_s^T: every block's local operator with its
                               snake terms (Sec. 2.3, Eqs. eq:DdagD / eq:diri) */
    DWF_OP_M5INV = 4,       /* M5op^-1 (dense Ls x Ls per chirality, Sec. 3.1.3) */
    DWF_OP_M5INVDAG = 5     /* (M5op^-1)^+ */
} dwf_op;

typedef struct {
    double tol;            /* stop when ||b - D^+D x|| / ||b|| <= tol (FP64, verified) */
    int maxiter;           /* outer iteration cap */
    int inner_iters;       /* k: fixed inner CG iterations of the preconditioner (Sec. 2.5) */
    dwf_prec outer_prec;   /* outer vectors: DWF_F64, DWF_F32, or DWF_F16 / DWF_BF16 / DWF_FX16 (16-bit
                              iterations as in Sec. 3.2; the solution increment stays FP32);
                              below FP64 with FP64 reliable updates */
    dwf_prec inner_prec;   /* DWF_F32, DWF_F16, DWF_BF16, DWF_FX16 or DWF_FX8 storage for the
                              inner solves */
    double delta;          /* reliable update when ||r|| < delta * max ||r|| since the last one */
    int use_reduced_ls;    /* 1: reduced-Ls preconditioner (dwf_set_reduced_ls first) */
    int use_graph;         /* 1: capture each outer iteration in a CUDA graph */
    int check_every;       /* the host reads the residual norm every check_every outer
                              iterations (<= 1: every one) and only then decides reliable
                              updates and convergence; the iterations in between run without
                              a host synchronisation (up to check_every - 1 extra iterations) */
    int time_kernels;      /* 1: time every operator application with CUDA events on the
                              solve's stream (reported in dwf_stats) */
    int precond_wave;      /* blocks whose k inner iterations run together (a "wave"):
                              0 = all blocks (default), > 0 = that many, < 0 = as many as
                              keep a wave's working set within half of L2 */
} dwf_solver_params;

typedef struct {
    int outer_iters;
    int inner_iters_total;
    int reliable_updates;
    int converged;
    double true_residual;     /* FP64 ||b - D^+D x|| / ||b|| at exit (per system for batches) */
    double time_total_ms;     /* device time of the solve (events on the handle's stream) */
    long long kernel_launches;/* kernels this call launched (graph nodes counted per replay) */
    double local_op_ms;       /* with time_kernels: summed device time of the local-operator
                                 applications of the preconditioner (4 hop stages each) */
    long long local_op_count;
    double outer_op_ms;       /* with time_kernels: summed device time of the outer D^+D */
    long long outer_op_count;
} dwf_stats;

/* Default parameters: tol 1e-10, maxiter 20000, k 6, FP32 outer, FP16 inner,
 * delta 0.1, no reduced Ls, graphs on, check every iteration. */
void dwf_default_params(dwf_solver_params *p);

/* Build a handle for one lattice.  dims[4] = (Lx, Ly, Lz, Lt), all even;
 * subdomain[4] = block dims (each even, divides dims[mu]; == dims[mu] means the
 * dimension is not partitioned; a partitioned dimension needs
 * dims[mu] - subdomain[mu] >= 4 so that no four-hop path leaves a block and
 * re-enters it from the far side).  subdomain may be NULL (one block).
 * b, c, M5, mass: Mobius parameters.  t_antiperiodic: 1 puts -1 on links that
 * cross the t boundary.  cuda_stream: the stream all work is issued on (0 =
 * legacy default stream).  Copies and compresses the gauge field. */
dwf_status dwf_create(dwf_handle **h, const double *gauge_host, const int dims[4], int Ls,
                      double b, double c, double M5, double mass, const int subdomain[4],
                      int t_antiperiodic, void *cuda_stream);
void dwf_destroy(dwf_handle *h);
const char *dwf_last_error(const dwf_handle *h);
const char *dwf_status_string(dwf_status s);

/* Number of elements (complex numbers) of a canonical even/odd field for this
 * handle with fifth extent Ls (0 = the handle's Ls). */
size_t dwf_field_elems(const dwf_handle *h, int Ls);
/* Bytes of the library's internal (packed) layout of one even field in
 * precision prec with fifth extent Ls (0 = the handle's Ls). */
size_t dwf_packed_bytes(const dwf_handle *h, dwf_prec prec, int Ls);

/* Site counts of the handle's geometry (all counts per parity; "padded"
 * counts are the device allocation sizes).  Local regions of one block
 * (Sec. 2.3, snake terms): interior = even sites of the block; o1 = odd sites
 * within one hop of it; e2 = even sites within two hops. */
typedef struct {
    long long even_sites;          /* V/2 */
    long long even_sites_padded;   /* packed field length in sites */
    long long blocks;
    long long block_sites, block_sites_padded;
    long long o1_sites, o1_sites_padded;
    long long e2_sites, e2_sites_padded;
} dwf_geometry;
dwf_status dwf_get_geometry(const dwf_handle *h, dwf_geometry *g);
/* The same counts for a lattice and block dims (same rules as dwf_create;
 * subdomain NULL = unpartitioned) without creating a handle or touching a
 * device: host-only, for sizing memory before dwf_create.  DWF_EINVAL for
 * dims or blocks dwf_create would refuse, DWF_EUNSUPPORTED for more than
 * 65535 blocks. */
dwf_status dwf_query_geometry(const int dims[4], const int subdomain[4], dwf_geometry *g);

/* Canonical <-> packed layout conversion on device buffers (stream 0 =
 * handle's stream).  Same precision on both sides. */
dwf_status dwf_pack(dwf_handle *h, void *packed_dev, const void *canonical_dev, dwf_prec prec,
                    void *stream);
dwf_status dwf_unpack(dwf_handle *h, void *canonical_dev, const void *packed_dev, dwf_prec prec,
                      void *stream);

/* out = op(in) on canonical even fields of precision prec (device buffers,
 * distinct).  FP64 and FP32 compute in their own precision; DWF_F16,
 * DWF_BF16 and DWF_FX16 store in 16 bits and compute in FP32, with the dense fifth-
 * dimension matrices on the tensor cores.  DWF_OP_LOCAL_DDAGD uses the
 * handle's block dims. */
dwf_status dwf_apply(dwf_handle *h, void *out_dev, const void *in_dev, dwf_op op, dwf_prec prec,
                     void *stream);
/* Same on packed fields (dwf_pack layout); no layout conversion. */
dwf_status dwf_apply_packed(dwf_handle *h, void *out_dev, const void *in_dev, dwf_op op,
                            dwf_prec prec, void *stream);

/* Plain CG (Algorithm 1 with M = 1, Fletcher-Reeves beta) on D^+D x = b.
 * x_dev, b_dev: canonical FP64 even fields; x_dev holds the initial guess. */
dwf_status dwf_cg(dwf_handle *h, double *x_dev, const double *b_dev, const dwf_solver_params *p,
                  dwf_stats *stats);
/* MSPCG (Algorithm 1, M = (+)_s A_s approximated by k inner CG iterations
 * from a zero guess, Polak-Ribiere beta, Sec. 3.2) on D^+D x = b. */
dwf_status dwf_mspcg(dwf_handle *h, double *x_dev, const double *b_dev,
                     const dwf_solver_params *p, dwf_stats *stats);
/* The same solves with HOST buffers: the call copies b in and x out. */
dwf_status dwf_solve_host(dwf_handle *h, double *x_host, const double *b_host,
                          const dwf_solver_params *p, int use_mspcg, dwf_stats *stats);

/* The preconditioner alone on a canonical FP64 even field: z = M^-1 r. */
dwf_status dwf_precondition(dwf_handle *h, double *z_dev, const double *r_dev,
                            const dwf_solver_params *p);

/* Reduced-Ls preconditioner (Sec. 3.3): z = (T^+ Mhat^-1 T + mu) r with Mhat
 * the local normal operator at Ls_hat (same b, c, M5, mass) and Mhat^-1 the
 * k-iteration inner CG.  T_host: (4*Ls_hat) x (4*Ls) complex (double[2]),
 * row index s*4 + spin, column index t*4 + spin; trivial in colour. */
dwf_status dwf_set_reduced_ls(dwf_handle *h, int Ls_hat, const double *T_host, double mu);

/* Training the reduced-Ls transform T (Sec. 3.3).  The loss
 *   chi^2(T) = sum_i | M (T^+ Mhat^-1 T + mu) v_i - v_i |^2
 * (M the local operator (+)_s A_s at Ls, Mhat the one at Ls_hat) and its
 * gradient are assembled from the three calls below plus dwf_apply with
 * DWF_OP_LOCAL_DDAGD; all fields are canonical even-checkerboard FP64 device
 * arrays of this handle's lattice (Ls or Ls_hat slices as stated).
 *
 * dwf_reduced_local_inverse: out = CG_iters(Mhat) in, x0 = 0, every block
 * independently (the inner solve of the preconditioner run to `iters`
 * iterations, standing in for Mhat^-1); p->inner_prec (FP32, FP16, BF16 or FX16;
 * the 16-bit formats need Ls_hat <= 16) sets the inner storage, p null means
 * dwf_default_params.  in, out: Ls_hat slices, out != in.
 *
 * dwf_apply_T: dagger = 0: out (Ls_hat slices) = T in (Ls slices);
 * dagger = 1: out (Ls slices) = T^+ in (Ls_hat slices).  T_host: (4 Ls_hat) x
 * (4 Ls) complex as double pairs, row s*4 + spin, column t*4 + spin, trivial in
 * colour (the layout of dwf_set_reduced_ls); applied in single precision.
 *
 * dwf_T_contract: G_host ((4 La) x (4 Lb) complex, double pairs, row-major) =
 * sum over sites x and colours c of a[s][x][spin][c] conj(b[t][x][spin'][c]),
 * row s*4 + spin, column t*4 + spin'; a has La slices, b has Lb slices,
 * 16 La Lb <= 4096.  Summed in FP64 in a fixed order (deterministic).
 *
 * All three synchronise the handle's stream before returning; DWF_EINVAL for
 * bad arguments, DWF_ECUDA / DWF_ENOMEM on device failures. */
dwf_status dwf_reduced_local_inverse(dwf_handle *h, double *out_dev, const double *in_dev, int Ls_hat,
                                     int iters, const dwf_solver_params *p);
dwf_status dwf_apply_T(dwf_handle *h, double *out_dev, const double *in_dev, const double *T_host,
                       int Ls_hat, int dagger);
dwf_status dwf_T_contract(dwf_handle *h, double *G_host, const double *a_dev, int La, const double *b_dev,
                          int Lb);

/* Vector arithmetic on canonical even-checkerboard fields of this handle's
 * lattice with Ls slices (0 = the handle's Ls), for callers that assemble
 * the method's outer loops (the transform training of Sec. 3.3) from the
 * library's operators.  Fields are device arrays of complex numbers, FP64
 * (DWF_F64) or FP32 (DWF_F32); both calls synchronise the handle's stream.
 *
 * dwf_field_axpby: out = a x + b y element by element, with the complex
 * coefficients a = (a_re, a_im), b = (b_re, b_im); x and y (y may be NULL:
 * out = a x, which with a = 1 converts between the precisions) in in_prec,
 * out in out_prec; out may be x or y when the precisions agree.
 *
 * dwf_field_dot: result_host[0] + i result_host[1] = sum conj(a_e) b_e,
 * accumulated in FP64 in a fixed order (the same inputs always give the same
 * bits).  DWF_EINVAL for null pointers or other precisions. */
dwf_status dwf_field_axpby(dwf_handle *h, void *out_dev, dwf_prec out_prec, double a_re, double a_im,
                           const void *x_dev, double b_re, double b_im, const void *y_dev, dwf_prec in_prec,
                           int Ls);
dwf_status dwf_field_dot(dwf_handle *h, double *result_host, const void *a_dev, const void *b_dev, dwf_prec prec,
                         int Ls);

/* Ablation of the snake terms (Sec. 2.3, Eq. (eq:diri)): with on != 0 every
 * later use of the local operator A_s on this handle (dwf_apply with
 * DWF_OP_LOCAL_DDAGD, dwf_precondition, dwf_mspcg) applies Dirichlet walls at
 * the block boundary on each of the four hops of D^+D instead of restricting
 * the full D^+D to the block, i.e. the truncated product on the left of
 * Eq. (eq:diri).  on = 0 restores A_s = R_s D^+D R_s^T.  The first call with
 * on != 0 builds the filtered neighbour tables on the device (DWF_ENOMEM or
 * DWF_ECUDA on failure).  Not part of the method: it exists to measure what
 * the snake terms buy. */
dwf_status dwf_set_local_truncated(dwf_handle *h, int on);

/* Batched MSPCG over independent lattices (uneven sizes allowed; same Ls,
 * b, c, M5 and block dims; per-lattice mass and gauge field).  The handles
 * stay owned by the caller and must outlive the batch. */
dwf_status dwf_batch_create(dwf_batch **bt, dwf_handle *const *hs, int n);
void dwf_batch_destroy(dwf_batch *bt);
/* xs[i], bs[i]: canonical FP64 even fields of system i (device).  per_system:
 * n stats (may be NULL); total: whole-batch stats (may be NULL). */
dwf_status dwf_batch_mspcg(dwf_batch *bt, double *const *xs, const double *const *bs,
                           const dwf_solver_params *p, dwf_stats *per_system, dwf_stats *total);

/* The global operators D, D^+ and D^+D (op as in dwf_apply) on packed fields,
 * with no device memory allocated by the call.  The paper has no counterpart;
 * this exists for callers that cannot allocate at this point (memory owned by
 * an arena or pool, no allocator calls allowed while other work is in flight,
 * hosts that forbid allocation after start-up).  The three intermediate fields
 * live in one file-scope device array of 24 MiB that every GPU which loads
 * this library holds until the process exits; lattices whose three fields in
 * this precision need more (3 x dwf_packed_bytes rounded up to 256 bytes)
 * are rejected with DWF_EINVAL.  Preconditions: one dwf_apply_packed call
 * with the same precision on this handle (it builds the link copies, the
 * fifth-dimension matrices and the launch configuration; this call never
 * does).  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  The address is kept for the life of the
 * process, so the entry point must not be used across a cudaDeviceReset (or a
 * release of the device's primary context).  Every call shares the one array,
 * so calls whose work overlaps on the GPU (other streams, other handles, other
 * threads) race; serialize them.  stream: 0 = the handle's stream. */
dwf_status dwf_apply_packed_static(dwf_handle *h, void *out_dev, const void *in_dev, dwf_op op,
                                   dwf_prec prec, void *stream);

/* Last error message of a batch. */
const char *dwf_batch_last_error(const dwf_batch *bt);

/* Launch configuration of the fused hop-stage kernels of one operator family
 * (op_kind 0: the global D, D^+, D^+D; 1: the local operator), in one
 * precision.  tile_sites: output 4D sites per CTA (each CTA holds their whole
 * Ls-slab); gather: 0 = neighbour spinors loaded by each thread, 1 = bulk
 * asynchronous copies (TMA engine) of whole neighbour Ls-columns into shared
 * memory, 2 = the hop itself on the tensor cores (16-bit storage only, 8-site
 * tiles, Ls in {4, 8, 12, 16}: per site the projected neighbour spinors,
 * rows (spin, slice) x columns (direction, colour), times the links, FP16
 * operands and FP32 accumulation).  By default the first use of an operator in a precision times every
 * candidate that fits and keeps the fastest (the autotuner, Sec. 3.1.3 tunes
 * block sizes the same way). */
typedef struct {
    int tile_sites;
    int gather;
} dwf_kernel_config;
dwf_status dwf_autotune(dwf_handle *h, dwf_prec prec, int op_kind);
dwf_status dwf_get_kernel_config(dwf_handle *h, dwf_prec prec, int op_kind, dwf_kernel_config *c);
/* Fix a configuration (disables autotuning for it).  Rejects choices that do
 * not fit (shared memory, threads, a tile that does not divide 32, the site
 * padding of every block and system) with DWF_EINVAL. */
dwf_status dwf_set_kernel_config(dwf_handle *h, dwf_prec prec, int op_kind,
                                 const dwf_kernel_config *c);

/* Bounded device waits.  The stage kernels that stage their neighbours with
 * bulk asynchronous copies (gather = 1 in dwf_kernel_config) wait for the
 * copies on an mbarrier; every such wait polls at most max_polls times
 * (max_polls <= 0: the default, 2^22) and then raises the handle's error flag,
 * which the next synchronising call (dwf_apply, the solvers) reports as
 * DWF_ETIMEOUT.  No wait ever traps or hangs.  force_timeout != 0 exists to
 * test that failure path: every such kernel then waits, after all of its
 * copies have landed, on a barrier phase that is never armed, so the wait runs
 * out with nothing in flight; 0 restores normal operation.  The handle stays
 * usable after a DWF_ETIMEOUT (the flag is cleared when it is reported). */
dwf_status dwf_set_wait_policy(dwf_handle *h, long long max_polls, int force_timeout);

/* Kernel launches issued by this library since load (process-wide). */
long long dwf_kernel_launch_count(void);

/* Measured fused multiply-add rate of the CUDA cores of the handle's device,
 * the compute roof of the FP32 stages and of the FP64 operator used by the
 * reliable updates (the roofline model of Sec. 3.1.1 needs the device's
 * peak rate).  prec: DWF_F32 or DWF_F64 (else DWF_EINVAL).  Runs one full
 * wave of independent FMA chains on the handle's stream (a warm-up and three
 * timed launches, a few ms each for FP32, ~15 ms for FP64), synchronises, and
 * writes the best rate in TFLOP/s (2 flops per FMA) to *tflops_host.
 * DWF_ECUDA on a CUDA error (dwf_last_error gives it). */
dwf_status dwf_fma_peak(dwf_handle *h, dwf_prec prec, double *tflops_host);

#ifdef __cplusplus
}
#endif
#endif
