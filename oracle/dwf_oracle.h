/*
 * Plain FP64 CPU oracle for the Mobius domain-wall operators and the
 * multi-splitting preconditioned CG of arXiv:2104.05615.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the bench's
 * CPU-baseline leg call it; the CUDA library never includes, links or calls
 * anything here, and nothing here includes the library's headers.
 *
 * Conventions (shared with the C ABI only through the documented layouts):
 *   complex numbers: C99 double _Complex
 *   site index     : lex = x + Lx*(y + Ly*(z + Lz*t)), parity = (x+y+z+t)%2
 *   full 5D field  : [Ls][V][4 spin][3 colour]
 *   even/odd field : [Ls][V/2][4][3], site index lex/2 among one parity
 *   gauge          : [V][4 mu][3][3], mu = x,y,z,t
 *   5D dense matrix: (4Ls)x(4Ls), row/column index s*4 + spin
 */
#ifndef DWF_ORACLE_H
#define DWF_ORACLE_H

#include <complex.h>

typedef double _Complex orc_c;

typedef struct {
    int L[4];            /* x, y, z, t extents */
    int Ls;              /* fifth-dimension extent */
    double b, c;         /* Mobius parameters */
    double M5;           /* domain-wall height */
    double mass;         /* quark mass on the wall wrap */
    int antiperiodic_t;  /* 1: links crossing the t boundary carry -1 */
} orc_params;

enum { ORC_P = 0, ORC_M5OP = 1, ORC_MPHI = 2, ORC_M5INV = 3 };
enum { ORC_PREC_NONE = 0, ORC_PREC_MSPCG = 1, ORC_PREC_REDUCED = 2 };
enum { ORC_BETA_FR = 0, ORC_BETA_PR = 1 };

/* gamma_{mu+1} for mu = 0..3 (x,y,z,t), gamma5 = g1 g2 g3 g4 for mu = 4;
 * row-major 4x4. */
void orc_gamma(int mu, orc_c *g);

/* D^w of Sec. 2.2 on the full lattice, every s slice; dagger=1 applies the
 * conjugate transpose, assembled term by term. */
void orc_hop(const orc_params *p, const orc_c *gauge, const orc_c *in,
             orc_c *out, int dagger);

/* Dense (4Ls)x(4Ls) fifth-dimension matrices: P (the chiral shift),
 * M5op = A + B P, M_phi = -(b + c P)/2, M5op^-1; dagger conjugate-transposes. */
void orc_5d_matrix(const orc_params *p, int which, int dagger, orc_c *M);
/* Apply a dense 5D matrix to every (4D site, colour) of a field with nsite
 * 4D sites, layout [Ls][nsite][4][3]. */
void orc_apply_5d(const orc_params *p, const orc_c *M, const orc_c *in,
                  orc_c *out, long nsite);
/* Closed form of the Ls x Ls block of M5op^-1 on chirality +1 or -1. */
void orc_m5inv_closed(const orc_params *p, int chirality, double *Minv);

/* Full (unpreconditioned) 5D operator M5op + D^w M_phi on full fields. */
void orc_D5(const orc_params *p, const orc_c *gauge, const orc_c *in,
            orc_c *out);
/* M^4 = D^w M_phi from parity `in_par` to the other parity (dagger: the
 * adjoint, from 1-in_par... see the source). even/odd layout. */
void orc_m4(const orc_params *p, const orc_c *gauge, const orc_c *in,
            int in_par, orc_c *out, int dagger);
/* Even-odd Schur operator D = 1 - M5^-1 M4_eo M5^-1 M4_oe (Sec. 2.2) and its
 * adjoint, on even fields. */
void orc_Deo(const orc_params *p, const orc_c *gauge, const orc_c *in,
             orc_c *out, int dagger);
void orc_DdagD(const orc_params *p, const orc_c *gauge, const orc_c *in,
               orc_c *out);
/* phi_hat_e = M5^-1 phi_e - M5^-1 M4_eo M5^-1 phi_o (phi full layout). */
void orc_phihat(const orc_params *p, const orc_c *gauge, const orc_c *phi,
                orc_c *out_e);
/* psi_o = M5^-1 (phi_o - M4_oe psi_e). */
void orc_reconstruct_odd(const orc_params *p, const orc_c *gauge,
                         const orc_c *psi_e, const orc_c *phi, orc_c *out_o);

/* Block index (0..nblock-1) of every even site for block dims sub[4]. */
long orc_block_ids(const orc_params *p, const int *sub, int *bid);
/* Local normal operator of every block: out = sum_s R_s^T (R_s D^+D R_s^T) R_s in
 * (Sec. 2.3: the local part of D^+D, snake terms included). */
void orc_local_DdagD(const orc_params *p, const orc_c *gauge, const int *sub,
                     const orc_c *in, orc_c *out);
/* Same, for one block only (output zero outside that block). */
void orc_local_DdagD_block(const orc_params *p, const orc_c *gauge,
                           const int *sub, long block, const orc_c *in,
                           orc_c *out);

/* Fifth-dimension transform of the reduced-Ls preconditioner (Sec. 3.4):
 * T is (4*Ls_hat) x (4*Ls) complex, row index s*4+spin; out has Ls_hat. */
void orc_T_apply(const orc_c *T, int Ls_hat, int Ls, long nsite,
                 const orc_c *in, orc_c *out, int dagger);

/* ||b - D^+D x|| / ||b|| in FP64. */
double orc_true_residual(const orc_params *p, const orc_c *gauge,
                         const orc_c *x, const orc_c *b);

typedef struct {
    int precond;        /* ORC_PREC_* */
    int beta;           /* ORC_BETA_* */
    int inner_iters;    /* k, fixed */
    int sub[4];         /* block dims */
    double tol;         /* relative residual */
    int maxiter;
    /* reduced-Ls preconditioner */
    int Ls_hat;
    const orc_c *T;
    double mu;
} orc_solver;

typedef struct {
    int iters;
    double true_res;
    int converged;
} orc_result;

/* Preconditioned CG of Algorithm 1 on D^+D x = b (even fields); x holds the
 * initial guess on entry.  res_hist (optional, maxiter+1 doubles) receives
 * ||r_k||/||b||. */
void orc_pcg(const orc_params *p, const orc_c *gauge, const orc_solver *sv,
             orc_c *x, const orc_c *b, orc_result *res, double *res_hist);
/* The preconditioner of Sec. 2.4 alone: z = (+)_s CG_k(A_s) r (or the
 * reduced-Ls form of Sec. 3.4). */
void orc_precond(const orc_params *p, const orc_c *gauge, const orc_solver *sv,
                 const orc_c *r, orc_c *z);

/* Threads the OpenMP runtime will use. */
int orc_num_threads(void);

#endif
