/*
 * Plain FP64 CPU oracle for arXiv:2104.05615 (Mobius domain-wall fermions,
 * multi-splitting preconditioned CG).
 *
 * TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the bench's
 * CPU baseline; never by the CUDA library.  Written for clarity, not speed:
 * every operator is assembled from its definition with full 4x4 gamma
 * matrices, full 3x3 links and dense (4Ls)x(4Ls) fifth-dimension matrices;
 * adjoints are literal conjugate transposes; even/odd blocks are obtained by
 * embedding into the full lattice and selecting a parity.
 *
 * Definitions followed (paper sections / equations):
 *   - D^w, the Wilson hopping term: Sec. 2.2, the equation defining D^w_{x,y}.
 *   - Even-odd block form, D = 1 - M5^-1 M4_eo M5^-1 M4_oe, phi_hat:
 *     Sec. 2.2, Eq. (dirac_equation); M4 = D^w M_phi: Sec. 2.2.
 *   - M5 and M_phi: the paper defers them to the Mobius formulation it cites
 *     (Sec. 2.2).  Reading used here (standard Mobius):
 *       D5 = (b D_W + 1) - (1 - c D_W) P,  D_W = (4 - M5) - D^w/2,
 *       (P psi)_s = P_- psi_{s+1} + P_+ psi_{s-1}, wrap terms times -mass,
 *     which splits exactly as D5 = M5op + D^w M_phi with
 *       M5op  = A + B P,  A = b(4-M5)+1,  B = c(4-M5)-1,
 *       M_phi = -(b + c P)/2.
 *     Gamma basis (paper silent): chiral DeGrand-Rossi, gamma5 =
 *     diag(-1,-1,+1,+1), P_+- = (1 +- gamma5)/2.
 *   - Normal equations D^+D: Sec. 2.2, Eq. (normal_equation).
 *   - Local operator with snake terms, A_s = R_s (D^+D) R_s^T: Sec. 2.3,
 *     Eqs. (eq:DdagD), (eq:diri); used as M = (+)_s A_s: Sec. 2.4.
 *   - Preconditioned CG: Algorithm 1 (alg:cg); fixed inner iteration count:
 *     Sec. 2.5; Polak-Ribiere beta: Sec. 3.2.
 *   - Reduced-Ls preconditioner z = (T^+ Mhat^-1 T + mu) r: Sec. 3.3.
 *
 * Pins (tests/test_oracle_*.py, all CPU): gamma algebra; dense brute force
 * against a textbook assembly of D5 on 2^4 x Ls=4; gamma5-hermiticity of D_W;
 * free-field plane-wave spectrum; M5op^-1 closed form vs elimination; gauge
 * covariance; Hermitian positivity of D^+D; even-odd Schur solve vs dense LU;
 * local operator vs an independent padded-field construction and vs the
 * truncated product; the FP64 true residual vs the dense matrix; the
 * preconditioner vs k textbook CG steps per dense block; CG/PCG identities;
 * the (s, spin) order of T by a selection matrix; reduced-Ls identities and
 * the reduced preconditioner as the composition of its parts.
 * Parity unpinned: outer iteration counts (the paper's ensembles are absent).
 */
#include "dwf_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NSC 12 /* spin x colour components per 5D site */

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

static long vol4(const orc_params *p)
{
    return (long)p->L[0] * p->L[1] * p->L[2] * p->L[3];
}

static void coords(const int *L, long lex, int *x)
{
    x[0] = (int)(lex % L[0]);
    lex /= L[0];
    x[1] = (int)(lex % L[1]);
    lex /= L[1];
    x[2] = (int)(lex % L[2]);
    x[3] = (int)(lex / L[2]);
}

static long lexi(const int *L, const int *x)
{
    return x[0] + (long)L[0] * (x[1] + (long)L[1] * (x[2] + (long)L[2] * x[3]));
}

static int parity_of(const int *x) { return (x[0] + x[1] + x[2] + x[3]) & 1; }

/* ------------------------------------------------------------------ gamma */

void orc_gamma(int mu, orc_c *g)
{
    /* Pauli matrices, row-major 2x2 */
    const orc_c s1[4] = {0, 1, 1, 0};
    const orc_c s2[4] = {0, -I, I, 0};
    const orc_c s3[4] = {1, 0, 0, -1};
    const orc_c *sig[3] = {s1, s2, s3};
    memset(g, 0, 16 * sizeof(orc_c));
    if (mu < 3) {
        /* gamma_k = [[0, i sigma_k], [-i sigma_k, 0]] */
        for (int a = 0; a < 2; a++)
            for (int b = 0; b < 2; b++) {
                g[a * 4 + (b + 2)] = I * sig[mu][a * 2 + b];
                g[(a + 2) * 4 + b] = -I * sig[mu][a * 2 + b];
            }
    } else if (mu == 3) {
        /* gamma_4 = [[0, 1], [1, 0]] */
        for (int a = 0; a < 2; a++) {
            g[a * 4 + (a + 2)] = 1;
            g[(a + 2) * 4 + a] = 1;
        }
    } else {
        /* gamma_5 = gamma_1 gamma_2 gamma_3 gamma_4 */
        orc_c acc[16], t[16], gm[16];
        orc_gamma(0, acc);
        for (int k = 1; k < 4; k++) {
            orc_gamma(k, gm);
            for (int i = 0; i < 4; i++)
                for (int j = 0; j < 4; j++) {
                    orc_c s = 0;
                    for (int l = 0; l < 4; l++) s += acc[i * 4 + l] * gm[l * 4 + j];
                    t[i * 4 + j] = s;
                }
            memcpy(acc, t, sizeof t);
        }
        memcpy(g, acc, sizeof acc);
    }
}

/* ------------------------------------------------------------ Wilson hop */

/* The 12x12 block of D^w coupling output site `site` to its neighbour
 * site + dir*mu (dir = +1: (1 - gamma_mu) U_{x,mu}; dir = -1:
 * (1 + gamma_mu) U^+_{x-mu,mu}), index spin*3 + colour. */
static void dw_block(const orc_params *p, const orc_c *gauge, long site,
                     int mu, int dir, orc_c *B)
{
    orc_c g[16], S[16], C[9];
    int x[4];
    double sign = 1.0;
    coords(p->L, site, x);
    orc_gamma(mu, g);
    for (int i = 0; i < 16; i++) S[i] = (i % 5 == 0 ? 1.0 : 0.0) - dir * g[i];
    if (dir > 0) {
        const orc_c *U = gauge + (site * 4 + mu) * 9;
        memcpy(C, U, sizeof C);
        if (p->antiperiodic_t && mu == 3 && x[3] == p->L[3] - 1) sign = -1.0;
    } else {
        int y[4] = {x[0], x[1], x[2], x[3]};
        y[mu] = (y[mu] - 1 + p->L[mu]) % p->L[mu];
        const orc_c *U = gauge + (lexi(p->L, y) * 4 + mu) * 9;
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) C[i * 3 + j] = conj(U[j * 3 + i]);
        if (p->antiperiodic_t && mu == 3 && x[3] == 0) sign = -1.0;
    }
    for (int a = 0; a < 4; a++)
        for (int i = 0; i < 3; i++)
            for (int b = 0; b < 4; b++)
                for (int j = 0; j < 3; j++)
                    B[(a * 3 + i) * NSC + (b * 3 + j)] = sign * S[a * 4 + b] * C[i * 3 + j];
}

static long neighbour(const orc_params *p, long site, int mu, int dir)
{
    int x[4];
    coords(p->L, site, x);
    x[mu] = (x[mu] + dir + p->L[mu]) % p->L[mu];
    return lexi(p->L, x);
}

void orc_hop(const orc_params *p, const orc_c *gauge, const orc_c *in,
             orc_c *out, int dagger)
{
    const long V = vol4(p);
    const int Ls = p->Ls;
#pragma omp parallel for schedule(static)
    for (long site = 0; site < V; site++) {
        orc_c B[8][NSC * NSC];
        long nb[8];
        for (int mu = 0; mu < 4; mu++)
            for (int d = 0; d < 2; d++) {
                int k = mu * 2 + d, dir = d ? -1 : 1;
                nb[k] = neighbour(p, site, mu, dir);
                if (!dagger) {
                    dw_block(p, gauge, site, mu, dir, B[k]);
                } else {
                    /* (D^w)^+_{x,y} = [(D^w)_{y,x}]^+ ; y reaches x in direction -dir */
                    orc_c T[NSC * NSC];
                    dw_block(p, gauge, nb[k], mu, -dir, T);
                    for (int i = 0; i < NSC; i++)
                        for (int j = 0; j < NSC; j++) B[k][i * NSC + j] = conj(T[j * NSC + i]);
                }
            }
        for (int s = 0; s < Ls; s++) {
            orc_c acc[NSC] = {0};
            for (int k = 0; k < 8; k++) {
                const orc_c *v = in + ((long)s * V + nb[k]) * NSC;
                for (int i = 0; i < NSC; i++) {
                    orc_c t = 0;
                    for (int j = 0; j < NSC; j++) t += B[k][i * NSC + j] * v[j];
                    acc[i] += t;
                }
            }
            memcpy(out + ((long)s * V + site) * NSC, acc, sizeof acc);
        }
    }
}

/* ------------------------------------------------- fifth-dimension matrices */

static void invert_dense(int n, orc_c *M)
{
    /* Gauss-Jordan elimination with partial pivoting, in place. */
    orc_c *A = malloc(sizeof(orc_c) * n * 2 * n);
    for (int i = 0; i < n; i++)
        for (int j = 0; j < 2 * n; j++)
            A[i * 2 * n + j] = j < n ? M[i * n + j] : (j - n == i ? 1.0 : 0.0);
    for (int col = 0; col < n; col++) {
        int piv = col;
        for (int r = col + 1; r < n; r++)
            if (cabs(A[r * 2 * n + col]) > cabs(A[piv * 2 * n + col])) piv = r;
        if (piv != col)
            for (int j = 0; j < 2 * n; j++) {
                orc_c t = A[col * 2 * n + j];
                A[col * 2 * n + j] = A[piv * 2 * n + j];
                A[piv * 2 * n + j] = t;
            }
        orc_c d = A[col * 2 * n + col];
        for (int j = 0; j < 2 * n; j++) A[col * 2 * n + j] /= d;
        for (int r = 0; r < n; r++) {
            if (r == col) continue;
            orc_c f = A[r * 2 * n + col];
            if (f == 0) continue;
            for (int j = 0; j < 2 * n; j++) A[r * 2 * n + j] -= f * A[col * 2 * n + j];
        }
    }
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) M[i * n + j] = A[i * 2 * n + n + j];
    free(A);
}

void orc_5d_matrix(const orc_params *p, int which, int dagger, orc_c *M)
{
    const int Ls = p->Ls, n = 4 * Ls;
    orc_c g5[16], Pp[16], Pm[16];
    orc_gamma(4, g5);
    for (int i = 0; i < 16; i++) {
        double id = (i % 5 == 0) ? 1.0 : 0.0;
        Pp[i] = 0.5 * (id + g5[i]);
        Pm[i] = 0.5 * (id - g5[i]);
    }
    orc_c *P = calloc((size_t)n * n, sizeof(orc_c));
    for (int s = 0; s < Ls; s++)
        for (int a = 0; a < 4; a++)
            for (int b = 0; b < 4; b++) {
                /* P_- psi_{s+1}, wrapping to s = 0 with -mass */
                if (s + 1 < Ls) P[(s * 4 + a) * n + (s + 1) * 4 + b] += Pm[a * 4 + b];
                else P[(s * 4 + a) * n + 0 * 4 + b] += -p->mass * Pm[a * 4 + b];
                /* P_+ psi_{s-1}, wrapping to s = Ls-1 with -mass */
                if (s - 1 >= 0) P[(s * 4 + a) * n + (s - 1) * 4 + b] += Pp[a * 4 + b];
                else P[(s * 4 + a) * n + (Ls - 1) * 4 + b] += -p->mass * Pp[a * 4 + b];
            }
    const double A = p->b * (4.0 - p->M5) + 1.0;
    const double Bc = p->c * (4.0 - p->M5) - 1.0;
    for (int i = 0; i < n * n; i++) {
        double id = (i / n == i % n) ? 1.0 : 0.0;
        switch (which) {
        case ORC_P: M[i] = P[i]; break;
        case ORC_M5OP:
        case ORC_M5INV: M[i] = A * id + Bc * P[i]; break;
        case ORC_MPHI: M[i] = -0.5 * (p->b * id + p->c * P[i]); break;
        }
    }
    free(P);
    if (which == ORC_M5INV) invert_dense(n, M);
    if (dagger) {
        for (int i = 0; i < n; i++)
            for (int j = i; j < n; j++) {
                orc_c a = M[i * n + j], b = M[j * n + i];
                M[i * n + j] = conj(b);
                M[j * n + i] = conj(a);
            }
    }
}

void orc_m5inv_closed(const orc_params *p, int chirality, double *Minv)
{
    const int Ls = p->Ls;
    const double A = p->b * (4.0 - p->M5) + 1.0;
    const double Bc = p->c * (4.0 - p->M5) - 1.0;
    const double q = -Bc / A, m = p->mass;
    const double den = A * (1.0 + m * pow(q, Ls));
    for (int s = 0; s < Ls; s++)
        for (int t = 0; t < Ls; t++) {
            /* chirality +1: lower cyclic shift; -1: its transpose */
            int a = chirality > 0 ? s : t, b = chirality > 0 ? t : s;
            int k = ((a - b) % Ls + Ls) % Ls;
            double f = (a >= b) ? 1.0 : -m;
            Minv[s * Ls + t] = pow(q, k) * f / den;
        }
}

void orc_apply_5d(const orc_params *p, const orc_c *M, const orc_c *in,
                  orc_c *out, long nsite)
{
    const int Ls = p->Ls, n = 4 * Ls;
#pragma omp parallel for schedule(static)
    for (long site = 0; site < nsite; site++)
        for (int col = 0; col < 3; col++) {
            orc_c v[4 * 64], w[4 * 64];
            for (int t = 0; t < Ls; t++)
                for (int b = 0; b < 4; b++) v[t * 4 + b] = in[(((long)t * nsite + site) * 4 + b) * 3 + col];
            for (int i = 0; i < n; i++) {
                orc_c acc = 0;
                for (int j = 0; j < n; j++) acc += M[i * n + j] * v[j];
                w[i] = acc;
            }
            for (int s = 0; s < Ls; s++)
                for (int a = 0; a < 4; a++) out[(((long)s * nsite + site) * 4 + a) * 3 + col] = w[s * 4 + a];
        }
}

static void apply_5d_named(const orc_params *p, int which, int dagger,
                           const orc_c *in, orc_c *out, long nsite)
{
    int n = 4 * p->Ls;
    orc_c *M = malloc(sizeof(orc_c) * n * n);
    orc_5d_matrix(p, which, dagger, M);
    orc_apply_5d(p, M, in, out, nsite);
    free(M);
}

/* ------------------------------------------------------- full 5D operator */

void orc_D5(const orc_params *p, const orc_c *gauge, const orc_c *in,
            orc_c *out)
{
    const long V = vol4(p), n = (long)p->Ls * V * NSC;
    orc_c *t = malloc(sizeof(orc_c) * n), *u = malloc(sizeof(orc_c) * n);
    apply_5d_named(p, ORC_MPHI, 0, in, t, V);
    orc_hop(p, gauge, t, u, 0);
    apply_5d_named(p, ORC_M5OP, 0, in, out, V);
    for (long i = 0; i < n; i++) out[i] += u[i];
    free(t);
    free(u);
}

/* ------------------------------------------------------------ even / odd */

static void embed(const orc_params *p, const orc_c *cb, int par, orc_c *full)
{
    const long V = vol4(p);
    memset(full, 0, sizeof(orc_c) * p->Ls * V * NSC);
    for (long lex = 0; lex < V; lex++) {
        int x[4];
        coords(p->L, lex, x);
        if (parity_of(x) != par) continue;
        for (int s = 0; s < p->Ls; s++)
            memcpy(full + ((long)s * V + lex) * NSC, cb + ((long)s * (V / 2) + lex / 2) * NSC,
                   sizeof(orc_c) * NSC);
    }
}

static void extract(const orc_params *p, const orc_c *full, int par, orc_c *cb)
{
    const long V = vol4(p);
    for (long lex = 0; lex < V; lex++) {
        int x[4];
        coords(p->L, lex, x);
        if (parity_of(x) != par) continue;
        for (int s = 0; s < p->Ls; s++)
            memcpy(cb + ((long)s * (V / 2) + lex / 2) * NSC, full + ((long)s * V + lex) * NSC,
                   sizeof(orc_c) * NSC);
    }
}

void orc_m4(const orc_params *p, const orc_c *gauge, const orc_c *in,
            int in_par, orc_c *out, int dagger)
{
    /* dagger = 0: out = (D^w M_phi)_{1-par, par} in
     * dagger = 1: out = [(D^w M_phi)_{par, 1-par}]^+ in = M_phi^+ (D^w)^+_{1-par,par} in */
    const long V = vol4(p), Vh = V / 2, nh = (long)p->Ls * Vh * NSC;
    orc_c *f1 = malloc(sizeof(orc_c) * 2 * nh), *f2 = malloc(sizeof(orc_c) * 2 * nh);
    orc_c *t = malloc(sizeof(orc_c) * nh);
    if (!dagger) {
        apply_5d_named(p, ORC_MPHI, 0, in, t, Vh);
        embed(p, t, in_par, f1);
        orc_hop(p, gauge, f1, f2, 0);
        extract(p, f2, 1 - in_par, out);
    } else {
        embed(p, in, in_par, f1);
        orc_hop(p, gauge, f1, f2, 1);
        extract(p, f2, 1 - in_par, t);
        apply_5d_named(p, ORC_MPHI, 1, t, out, Vh);
    }
    free(f1);
    free(f2);
    free(t);
}

void orc_Deo(const orc_params *p, const orc_c *gauge, const orc_c *in,
             orc_c *out, int dagger)
{
    const long Vh = vol4(p) / 2, nh = (long)p->Ls * Vh * NSC;
    orc_c *t = malloc(sizeof(orc_c) * nh), *u = malloc(sizeof(orc_c) * nh);
    if (!dagger) {
        /* D x = x - M5^-1 M4_eo M5^-1 M4_oe x */
        orc_m4(p, gauge, in, 0, t, 0);
        apply_5d_named(p, ORC_M5INV, 0, t, u, Vh);
        orc_m4(p, gauge, u, 1, t, 0);
        apply_5d_named(p, ORC_M5INV, 0, t, u, Vh);
    } else {
        /* D^+ x = x - M4_oe^+ M5^-+ M4_eo^+ M5^-+ x */
        apply_5d_named(p, ORC_M5INV, 1, in, t, Vh);
        orc_m4(p, gauge, t, 0, u, 1);
        apply_5d_named(p, ORC_M5INV, 1, u, t, Vh);
        orc_m4(p, gauge, t, 1, u, 1);
    }
    for (long i = 0; i < nh; i++) out[i] = in[i] - u[i];
    free(t);
    free(u);
}

void orc_DdagD(const orc_params *p, const orc_c *gauge, const orc_c *in,
               orc_c *out)
{
    const long nh = (long)p->Ls * (vol4(p) / 2) * NSC;
    orc_c *t = malloc(sizeof(orc_c) * nh);
    orc_Deo(p, gauge, in, t, 0);
    orc_Deo(p, gauge, t, out, 1);
    free(t);
}

void orc_phihat(const orc_params *p, const orc_c *gauge, const orc_c *phi,
                orc_c *out_e)
{
    const long Vh = vol4(p) / 2, nh = (long)p->Ls * Vh * NSC;
    orc_c *pe = malloc(sizeof(orc_c) * nh), *po = malloc(sizeof(orc_c) * nh);
    orc_c *t = malloc(sizeof(orc_c) * nh), *u = malloc(sizeof(orc_c) * nh);
    extract(p, phi, 0, pe);
    extract(p, phi, 1, po);
    apply_5d_named(p, ORC_M5INV, 0, po, t, Vh);
    orc_m4(p, gauge, t, 1, u, 0);
    for (long i = 0; i < nh; i++) pe[i] -= u[i];
    apply_5d_named(p, ORC_M5INV, 0, pe, out_e, Vh);
    free(pe);
    free(po);
    free(t);
    free(u);
}

void orc_reconstruct_odd(const orc_params *p, const orc_c *gauge,
                         const orc_c *psi_e, const orc_c *phi, orc_c *out_o)
{
    const long Vh = vol4(p) / 2, nh = (long)p->Ls * Vh * NSC;
    orc_c *po = malloc(sizeof(orc_c) * nh), *t = malloc(sizeof(orc_c) * nh);
    extract(p, phi, 1, po);
    orc_m4(p, gauge, psi_e, 0, t, 0);
    for (long i = 0; i < nh; i++) po[i] -= t[i];
    apply_5d_named(p, ORC_M5INV, 0, po, out_o, Vh);
    free(po);
    free(t);
}

/* -------------------------------------------------------- local operator */

long orc_block_ids(const orc_params *p, const int *sub, int *bid)
{
    const long V = vol4(p);
    int nb[4];
    for (int mu = 0; mu < 4; mu++) nb[mu] = p->L[mu] / sub[mu];
    for (long lex = 0; lex < V; lex++) {
        int x[4];
        coords(p->L, lex, x);
        if (parity_of(x) != 0) continue;
        long b = x[0] / sub[0] + (long)nb[0] * (x[1] / sub[1] + (long)nb[1] * (x[2] / sub[2] + (long)nb[2] * (x[3] / sub[3])));
        bid[lex / 2] = (int)b;
    }
    return (long)nb[0] * nb[1] * nb[2] * nb[3];
}

void orc_local_DdagD_block(const orc_params *p, const orc_c *gauge,
                           const int *sub, long block, const orc_c *in,
                           orc_c *out)
{
    const long Vh = vol4(p) / 2, nh = (long)p->Ls * Vh * NSC;
    int *bid = malloc(sizeof(int) * Vh);
    orc_block_ids(p, sub, bid);
    orc_c *t = calloc(nh, sizeof(orc_c)), *u = malloc(sizeof(orc_c) * nh);
    for (int s = 0; s < p->Ls; s++)
        for (long i = 0; i < Vh; i++)
            if (bid[i] == block) memcpy(t + ((long)s * Vh + i) * NSC, in + ((long)s * Vh + i) * NSC, sizeof(orc_c) * NSC);
    orc_DdagD(p, gauge, t, u);
    for (int s = 0; s < p->Ls; s++)
        for (long i = 0; i < Vh; i++) {
            orc_c *o = out + ((long)s * Vh + i) * NSC;
            if (bid[i] == block) memcpy(o, u + ((long)s * Vh + i) * NSC, sizeof(orc_c) * NSC);
            else memset(o, 0, sizeof(orc_c) * NSC);
        }
    free(bid);
    free(t);
    free(u);
}

void orc_local_DdagD(const orc_params *p, const orc_c *gauge, const int *sub,
                     const orc_c *in, orc_c *out)
{
    const long Vh = vol4(p) / 2, nh = (long)p->Ls * Vh * NSC;
    int *bid = malloc(sizeof(int) * Vh);
    long nblock = orc_block_ids(p, sub, bid);
    orc_c *u = malloc(sizeof(orc_c) * nh);
    memset(out, 0, sizeof(orc_c) * nh);
    for (long blk = 0; blk < nblock; blk++) {
        orc_local_DdagD_block(p, gauge, sub, blk, in, u);
        for (long i = 0; i < nh; i++) out[i] += u[i];
    }
    free(bid);
    free(u);
}

/* ------------------------------------------------------- reduced-Ls map */

void orc_T_apply(const orc_c *T, int Ls_hat, int Ls, long nsite,
                 const orc_c *in, orc_c *out, int dagger)
{
    const int nr = 4 * Ls_hat, nc = 4 * Ls;
    const int Lin = dagger ? Ls_hat : Ls, Lout = dagger ? Ls : Ls_hat;
#pragma omp parallel for schedule(static)
    for (long site = 0; site < nsite; site++)
        for (int col = 0; col < 3; col++) {
            orc_c v[4 * 64];
            for (int t = 0; t < Lin; t++)
                for (int b = 0; b < 4; b++) v[t * 4 + b] = in[(((long)t * nsite + site) * 4 + b) * 3 + col];
            for (int s = 0; s < Lout; s++)
                for (int a = 0; a < 4; a++) {
                    orc_c acc = 0;
                    int i = s * 4 + a;
                    if (!dagger)
                        for (int j = 0; j < nc; j++) acc += T[i * nc + j] * v[j];
                    else
                        for (int j = 0; j < nr; j++) acc += conj(T[j * nc + i]) * v[j];
                    out[(((long)s * nsite + site) * 4 + a) * 3 + col] = acc;
                }
        }
}

/* ------------------------------------------------------------- solvers */

static orc_c dotc(const orc_c *a, const orc_c *b, long n)
{
    double re = 0, im = 0;
#pragma omp parallel for reduction(+ : re, im) schedule(static)
    for (long i = 0; i < n; i++) {
        orc_c t = conj(a[i]) * b[i];
        re += creal(t);
        im += cimag(t);
    }
    return re + I * im;
}

double orc_true_residual(const orc_params *p, const orc_c *gauge,
                         const orc_c *x, const orc_c *b)
{
    const long nh = (long)p->Ls * (vol4(p) / 2) * NSC;
    orc_c *Ax = malloc(sizeof(orc_c) * nh);
    orc_DdagD(p, gauge, x, Ax);
    for (long i = 0; i < nh; i++) Ax[i] = b[i] - Ax[i];
    double r = sqrt(creal(dotc(Ax, Ax, nh))), bn = sqrt(creal(dotc(b, b, nh)));
    free(Ax);
    return r / bn;
}

/* Real part of per-block inner products <a,b>_blk over even fields. */
static void block_dots(const orc_c *a, const orc_c *b, const int *bid, long nblock,
                       int Ls, long Vh, double *out)
{
    for (long k = 0; k < nblock; k++) out[k] = 0;
    for (int s = 0; s < Ls; s++)
        for (long i = 0; i < Vh; i++) {
            const orc_c *x = a + ((long)s * Vh + i) * NSC, *y = b + ((long)s * Vh + i) * NSC;
            double acc = 0;
            for (int j = 0; j < NSC; j++) acc += creal(conj(x[j]) * y[j]);
            out[bid[i]] += acc;
        }
}

/* k plain CG iterations on M = (+)_s A_s from a zero guess, every block with
 * its own alpha, beta (Sec. 2.4-2.5).  An exact zero residual stops a block. */
static void inner_cg(const orc_params *p, const orc_c *gauge, const int *sub,
                     int k, const orc_c *r_in, orc_c *z)
{
    const long Vh = vol4(p) / 2, nh = (long)p->Ls * Vh * NSC;
    int *bid = malloc(sizeof(int) * Vh);
    long nblock = orc_block_ids(p, sub, bid);
    orc_c *r = malloc(sizeof(orc_c) * nh), *pv = malloc(sizeof(orc_c) * nh);
    orc_c *Ap = malloc(sizeof(orc_c) * nh);
    double *rr = malloc(sizeof(double) * nblock), *pAp = malloc(sizeof(double) * nblock);
    double *rr_new = malloc(sizeof(double) * nblock);
    double *alpha = malloc(sizeof(double) * nblock), *beta = malloc(sizeof(double) * nblock);
    memcpy(r, r_in, sizeof(orc_c) * nh);
    memcpy(pv, r_in, sizeof(orc_c) * nh);
    memset(z, 0, sizeof(orc_c) * nh);
    block_dots(r, r, bid, nblock, p->Ls, Vh, rr);
    for (int it = 0; it < k; it++) {
        orc_local_DdagD(p, gauge, sub, pv, Ap);
        block_dots(pv, Ap, bid, nblock, p->Ls, Vh, pAp);
        for (long q = 0; q < nblock; q++) alpha[q] = (rr[q] != 0 && pAp[q] != 0) ? rr[q] / pAp[q] : 0.0;
        for (int s = 0; s < p->Ls; s++)
            for (long i = 0; i < Vh; i++) {
                double a = alpha[bid[i]];
                long o = ((long)s * Vh + i) * NSC;
                for (int j = 0; j < NSC; j++) {
                    z[o + j] += a * pv[o + j];
                    r[o + j] -= a * Ap[o + j];
                }
            }
        block_dots(r, r, bid, nblock, p->Ls, Vh, rr_new);
        for (long q = 0; q < nblock; q++) beta[q] = rr[q] != 0 ? rr_new[q] / rr[q] : 0.0;
        for (int s = 0; s < p->Ls; s++)
            for (long i = 0; i < Vh; i++) {
                double bta = beta[bid[i]];
                long o = ((long)s * Vh + i) * NSC;
                for (int j = 0; j < NSC; j++) pv[o + j] = r[o + j] + bta * pv[o + j];
            }
        memcpy(rr, rr_new, sizeof(double) * nblock);
    }
    free(bid);
    free(r);
    free(pv);
    free(Ap);
    free(rr);
    free(pAp);
    free(rr_new);
    free(alpha);
    free(beta);
}

void orc_precond(const orc_params *p, const orc_c *gauge, const orc_solver *sv,
                 const orc_c *r, orc_c *z)
{
    const long Vh = vol4(p) / 2, nh = (long)p->Ls * Vh * NSC;
    if (sv->precond == ORC_PREC_NONE) {
        memcpy(z, r, sizeof(orc_c) * nh);
    } else if (sv->precond == ORC_PREC_MSPCG) {
        inner_cg(p, gauge, sv->sub, sv->inner_iters, r, z);
    } else {
        /* z = (T^+ Mhat^-1 T + mu) r, Mhat the local operator at Ls_hat */
        orc_params ph = *p;
        ph.Ls = sv->Ls_hat;
        const long nhh = (long)sv->Ls_hat * Vh * NSC;
        orc_c *rh = malloc(sizeof(orc_c) * nhh), *zh = malloc(sizeof(orc_c) * nhh);
        orc_T_apply(sv->T, sv->Ls_hat, p->Ls, Vh, r, rh, 0);
        inner_cg(&ph, gauge, sv->sub, sv->inner_iters, rh, zh);
        orc_T_apply(sv->T, sv->Ls_hat, p->Ls, Vh, zh, z, 1);
        for (long i = 0; i < nh; i++) z[i] += sv->mu * r[i];
        free(rh);
        free(zh);
    }
}

void orc_pcg(const orc_params *p, const orc_c *gauge, const orc_solver *sv,
             orc_c *x, const orc_c *b, orc_result *res, double *res_hist)
{
    const long nh = (long)p->Ls * (vol4(p) / 2) * NSC;
    orc_c *r = malloc(sizeof(orc_c) * nh), *z = malloc(sizeof(orc_c) * nh);
    orc_c *pv = malloc(sizeof(orc_c) * nh), *Ap = malloc(sizeof(orc_c) * nh);
    orc_c *r_old = malloc(sizeof(orc_c) * nh);
    const double bnorm = sqrt(creal(dotc(b, b, nh)));
    /* r0 = b - A x0, z0 = M^-1 r0, p0 = z0 */
    orc_DdagD(p, gauge, x, Ap);
    for (long i = 0; i < nh; i++) r[i] = b[i] - Ap[i];
    orc_precond(p, gauge, sv, r, z);
    memcpy(pv, z, sizeof(orc_c) * nh);
    double rz = creal(dotc(r, z, nh));
    double rnorm = sqrt(creal(dotc(r, r, nh)));
    if (res_hist) res_hist[0] = rnorm / bnorm;
    int k = 0, conv = rnorm / bnorm < sv->tol;
    while (!conv && k < sv->maxiter) {
        orc_DdagD(p, gauge, pv, Ap);
        double pAp = creal(dotc(pv, Ap, nh));
        double alpha = rz / pAp;
        memcpy(r_old, r, sizeof(orc_c) * nh);
        for (long i = 0; i < nh; i++) {
            x[i] += alpha * pv[i];
            r[i] -= alpha * Ap[i];
        }
        orc_precond(p, gauge, sv, r, z);
        double rz_new = creal(dotc(z, r, nh));
        double beta;
        if (sv->beta == ORC_BETA_PR) {
            for (long i = 0; i < nh; i++) r_old[i] = r[i] - r_old[i];
            beta = creal(dotc(z, r_old, nh)) / rz;
        } else {
            beta = rz_new / rz;
        }
        for (long i = 0; i < nh; i++) pv[i] = z[i] + beta * pv[i];
        rz = rz_new;
        k++;
        rnorm = sqrt(creal(dotc(r, r, nh)));
        if (res_hist) res_hist[k] = rnorm / bnorm;
        conv = rnorm / bnorm < sv->tol;
    }
    res->iters = k;
    res->true_res = orc_true_residual(p, gauge, x, b);
    res->converged = conv;
    free(r);
    free(z);
    free(pv);
    free(Ap);
    free(r_old);
}
