"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test is chosen so that a plausible mistake in the oracle (a wrong gamma
entry, a dropped hop term, a wrong sign, a transposed 5D matrix, a misplaced
mass wrap, a broken even/odd embedding, a wrong adjoint) fails at least one.
"""
import numpy as np
import pytest

from paper_2104_05615_gb300 import inputs
from tests.helpers_dense import (G, G5, PMINUS, PPLUS, coords, dense_of, gauge_transform,
                                 lexi, mobius_d5_textbook, parity_index)

PAR = dict(b=1.5, c=0.5, M5=1.8)


def make(orc, dims, Ls, mass=0.05, eps=0.5, seed=11, anti=0):
    U = inputs.gauge_field(dims, eps, seed)
    return orc.Oracle(dims, Ls, PAR["b"], PAR["c"], PAR["M5"], mass, U, anti), U


def rnd(shape, seed):
    r = np.random.default_rng(seed)
    return r.standard_normal(shape) + 1j * r.standard_normal(shape)


# --------------------------------------------------------------- gamma


def test_gamma_matrices_clifford_and_chiral(orc):
    gs = [orc.gamma(mu) for mu in range(4)]
    for mu in range(4):
        np.testing.assert_allclose(gs[mu], G[mu], atol=0)
        for nu in range(4):
            ac = gs[mu] @ gs[nu] + gs[nu] @ gs[mu]
            np.testing.assert_allclose(ac, 2 * np.eye(4) * (mu == nu), atol=1e-15)
    g5 = orc.gamma(4)
    np.testing.assert_allclose(g5, G5, atol=1e-15)
    for mu in range(4):
        np.testing.assert_allclose(g5 @ gs[mu] + gs[mu] @ g5, 0, atol=1e-15)


# ---------------------------------------------------- dense brute force


@pytest.mark.parametrize("anti", [0, 1])
def test_D5_matches_textbook_mobius_dense(orc, anti):
    """M5op + D^w M_phi (oracle) == (b D_W + 1) - (1 - c D_W) P (textbook), 2^4 x Ls=4."""
    dims, Ls, mass = (2, 2, 2, 2), 4, 0.07
    o, U = make(orc, dims, Ls, mass=mass, anti=anti)
    Ueff = U.copy()
    if anti:  # antiperiodic t: links crossing the t boundary flip sign
        for lex in range(16):
            if coords(dims, lex)[3] == dims[3] - 1:
                Ueff[lex, 3] *= -1
    D_or = dense_of(o.D5, o.full_shape())
    D_tb = mobius_d5_textbook(Ueff, dims, Ls, PAR["b"], PAR["c"], PAR["M5"], mass)
    np.testing.assert_allclose(D_or, D_tb, atol=1e-13)


def test_hop_adjoint_is_conjugate_transpose(orc):
    o, _ = make(orc, (4, 2, 2, 4), 3)
    x, y = rnd(o.full_shape(), 1), rnd(o.full_shape(), 2)
    lhs = np.vdot(y, o.hop(x))
    rhs = np.vdot(o.hop(y, dagger=True), x)
    assert abs(lhs - rhs) < 1e-11 * abs(lhs)


def test_Deo_adjoint_and_DdagD_hermitian_positive(orc):
    dims, Ls = (2, 2, 2, 2), 4
    o, _ = make(orc, dims, Ls)
    D = dense_of(o.D, o.cb_shape())
    Dd = dense_of(lambda v: o.D(v, dagger=True), o.cb_shape())
    np.testing.assert_allclose(Dd, D.conj().T, atol=1e-13)
    A = dense_of(o.DdagD, o.cb_shape())
    np.testing.assert_allclose(A, A.conj().T, atol=1e-12)
    ev = np.linalg.eigvalsh(A)
    assert ev.min() > 0
    np.testing.assert_allclose(A, D.conj().T @ D, atol=1e-12)


def test_gamma5_hermiticity_of_wilson(orc):
    """gamma5 D^w gamma5 = (D^w)^+ (so D_W is gamma5-hermitian)."""
    o, _ = make(orc, (4, 2, 4, 2), 2)
    x = rnd(o.full_shape(), 3)
    g5x = np.einsum("ab,svbc->svac", G5, x)
    lhs = np.einsum("ab,svbc->svac", G5, o.hop(g5x))
    np.testing.assert_allclose(lhs, o.hop(x, dagger=True), atol=1e-12)


def test_shamir_reflection_hermiticity(orc):
    """Shamir (b=1, c=0): Gamma5 R5 D5 Gamma5 R5 = D5^+."""
    dims, Ls = (2, 2, 2, 2), 4
    U = inputs.gauge_field(dims, 0.5, 5)
    o = orc.Oracle(dims, Ls, 1.0, 0.0, 1.8, 0.1, U)
    D = dense_of(o.D5, o.full_shape())
    V = 16
    R = np.kron(np.fliplr(np.eye(Ls)), np.kron(np.eye(V), np.kron(G5, np.eye(3))))
    np.testing.assert_allclose(R @ D @ R, D.conj().T, atol=1e-13)


# ----------------------------------------------------------- free field


def test_free_field_plane_waves(orc):
    """U = 1: D^w e^{ipx} chi = sum_mu [2 cos p_mu - 2 i gamma_mu sin p_mu] e^{ipx} chi."""
    dims, Ls = (4, 4, 2, 6), 1
    V = int(np.prod(dims))
    U = np.broadcast_to(np.eye(3), (V, 4, 3, 3)).copy()
    o = orc.Oracle(dims, Ls, 1.5, 0.5, 1.8, 0.0, U)
    rng = np.random.default_rng(0)
    for trial in range(4):
        n = [rng.integers(0, L) for L in dims]
        p = [2 * np.pi * n[m] / dims[m] for m in range(4)]
        chi = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
        psi = np.zeros((1, V, 4, 3), dtype=np.complex128)
        for lex in range(V):
            x = coords(dims, lex)
            psi[0, lex] = np.exp(1j * sum(p[m] * x[m] for m in range(4))) * chi
        K = sum(2 * np.cos(p[m]) * np.eye(4) - 2j * np.sin(p[m]) * G[m] for m in range(4))
        expect = np.einsum("ab,vbc->vac", K, psi[0])
        np.testing.assert_allclose(o.hop(psi)[0], expect, atol=1e-12)


def test_free_field_5d_spectrum(orc):
    """Singular values of the dense oracle D5 (U = 1) equal the union over momenta
    of those of the 4Ls x 4Ls textbook D5(p)."""
    dims, Ls, mass = (4, 2, 2, 2), 3, 0.1
    V = int(np.prod(dims))
    U = np.broadcast_to(np.eye(3), (V, 4, 3, 3)).copy()
    o = orc.Oracle(dims, Ls, 1.5, 0.5, 1.8, mass, U)
    sv_or = np.sort(np.linalg.svd(dense_of(o.D5, o.full_shape()), compute_uv=False))
    Eup = np.diag(np.ones(Ls - 1), 1); Eup[Ls - 1, 0] = -mass
    Edn = np.diag(np.ones(Ls - 1), -1); Edn[0, Ls - 1] = -mass
    P = np.kron(Eup, PMINUS) + np.kron(Edn, PPLUS)
    svs = []
    import itertools
    for n in itertools.product(*[range(L) for L in dims]):
        p = [2 * np.pi * n[m] / dims[m] for m in range(4)]
        DW = (4 - 1.8 - sum(np.cos(p))) * np.eye(4) + 1j * sum(G[m] * np.sin(p[m]) for m in range(4))
        I5 = np.eye(Ls)
        Dp = np.kron(I5, 1.5 * DW + np.eye(4))
        Dm = np.kron(I5, np.eye(4) - 0.5 * DW)
        Dp5 = Dp - Dm @ P
        s = np.linalg.svd(Dp5, compute_uv=False)
        svs.extend(list(s) * 3)  # colour multiplicity
    np.testing.assert_allclose(sv_or, np.sort(svs), atol=1e-12)


# ------------------------------------------------------------ M5 inverse


@pytest.mark.parametrize("Ls,mass", [(4, 0.1), (8, 0.01), (12, 0.002), (16, 0.001)])
def test_m5inv_closed_form_and_elimination(orc, Ls, mass):
    o, _ = make(orc, (2, 2, 2, 2), Ls, mass=mass)
    M = o.matrix5(orc.M5OP)
    Mi = o.matrix5(orc.M5INV)
    np.testing.assert_allclose(M @ Mi, np.eye(4 * Ls), atol=1e-14)
    # chirality blocks: spins 2,3 are chirality +1, spins 0,1 are -1
    for chir, spin in [(+1, 2), (-1, 0)]:
        blk = Mi[spin::4, spin::4].real
        np.testing.assert_allclose(blk, o.m5inv_closed(chir), atol=1e-14)
        assert np.abs(Mi[spin::4, spin::4].imag).max() == 0
    # no chirality mixing
    assert np.abs(Mi[0::4, 2::4]).max() == 0 and np.abs(Mi[2::4, 1::4]).max() == 0
    Md = o.matrix5(orc.M5INV, dagger=True)
    np.testing.assert_allclose(Md, Mi.conj().T, atol=0)


def test_5d_op_structure(orc):
    """M5op and M_phi commute; M_phi = -(b + c P)/2 and M5op = A + B P."""
    o, _ = make(orc, (2, 2, 2, 2), 6, mass=0.03)
    P = o.matrix5(orc.P)
    A = 1.5 * (4 - 1.8) + 1
    B = 0.5 * (4 - 1.8) - 1
    np.testing.assert_allclose(o.matrix5(orc.M5OP), A * np.eye(24) + B * P, atol=1e-15)
    Mp = o.matrix5(orc.MPHI)
    np.testing.assert_allclose(Mp, -0.5 * (1.5 * np.eye(24) + 0.5 * P), atol=1e-15)
    M5 = o.matrix5(orc.M5OP)
    np.testing.assert_allclose(M5 @ Mp, Mp @ M5, atol=1e-14)


# ------------------------------------------------------- gauge covariance


def test_gauge_covariance(orc):
    dims, Ls = (4, 2, 2, 4), 3
    o, U = make(orc, dims, Ls, eps=0.8)
    V = int(np.prod(dims))
    g = inputs.random_su3(V, 77)
    o2 = orc.Oracle(dims, Ls, 1.5, 0.5, 1.8, 0.05, gauge_transform(U, g, dims))
    x = rnd(o.full_shape(), 9)
    gx = np.einsum("vij,svaj->svai", g, x)
    np.testing.assert_allclose(o2.hop(gx), np.einsum("vij,svaj->svai", g, o.hop(x)), atol=1e-12)
    # even/odd normal operator and the local operator are covariant too
    xe = rnd(o.cb_shape(), 10)
    ge = np.empty((V // 2, 3, 3), dtype=np.complex128)
    for lex in range(V):
        if sum(coords(dims, lex)) % 2 == 0:
            ge[lex // 2] = g[lex]
    gxe = np.einsum("vij,svaj->svai", ge, xe)
    np.testing.assert_allclose(o2.DdagD(gxe), np.einsum("vij,svaj->svai", ge, o.DdagD(xe)),
                               atol=1e-11)
    sub = (4, 2, 2, 2)
    np.testing.assert_allclose(o2.local_DdagD(gxe, sub),
                               np.einsum("vij,svaj->svai", ge, o.local_DdagD(xe, sub)), atol=1e-11)


# -------------------------------------------------------- even-odd Schur


def test_even_odd_schur_solve_matches_full_solve(orc):
    dims, Ls = (2, 2, 2, 2), 4
    o, _ = make(orc, dims, Ls, mass=0.1)
    D5 = dense_of(o.D5, o.full_shape())
    phi = rnd(o.full_shape(), 4)
    psi = np.linalg.solve(D5, phi.reshape(-1))
    Deo = dense_of(o.D, o.cb_shape())
    psi_e = np.linalg.solve(Deo, o.phihat(phi).reshape(-1)).reshape(o.cb_shape())
    psi_o = o.reconstruct_odd(psi_e, phi)
    ie, io = parity_index(dims, Ls, 0), parity_index(dims, Ls, 1)
    np.testing.assert_allclose(psi_e.reshape(-1), psi[ie], atol=1e-11)
    np.testing.assert_allclose(psi_o.reshape(-1), psi[io], atol=1e-11)


def test_schur_block_form(orc):
    """The dense D5 restricted to parities has M5op on the diagonal blocks and
    M4 = D^w M_phi on the off-diagonal ones (the paper's block form)."""
    dims, Ls = (2, 2, 2, 2), 3
    o, _ = make(orc, dims, Ls)
    D5 = dense_of(o.D5, o.full_shape())
    ie, io = parity_index(dims, Ls, 0), parity_index(dims, Ls, 1)
    M4oe = dense_of(lambda v: o.m4(v, 0), o.cb_shape())
    M4eo = dense_of(lambda v: o.m4(v, 1), o.cb_shape())
    np.testing.assert_allclose(D5[np.ix_(io, ie)], M4oe, atol=1e-13)
    np.testing.assert_allclose(D5[np.ix_(ie, io)], M4eo, atol=1e-13)
    M5 = o.matrix5(orc.M5OP)
    blk = D5[np.ix_(ie, ie)]
    e5 = o.apply5(M5, np.eye(blk.shape[0]).T.reshape((blk.shape[0],) + o.cb_shape())[0])
    np.testing.assert_allclose(blk[:, 0], e5.reshape(-1), atol=1e-14)
    # adjoint M4 (dagger flag) is the conjugate transpose
    M4oe_d = dense_of(lambda v: o.m4(v, 1, dagger=True), o.cb_shape())
    np.testing.assert_allclose(M4oe_d, M4oe.conj().T, atol=1e-13)


# ------------------------------------------------- local operator (snakes)


def _padded_local(o, dims, Ls, sub, origin, pad):
    """Independent construction of the paper's padded-field method (Sec. 3.1.2):
    zero-padded block, the four hops applied with Dirichlet walls at the pad edge."""
    V = int(np.prod(dims))
    def in_region(lex, width):
        x = coords(dims, lex)
        for mu in range(4):
            if sub[mu] == dims[mu]:
                continue
            d = (x[mu] - origin[mu]) % dims[mu]
            lo, hi = -width, sub[mu] - 1 + width
            dd = d if d <= hi else d - dims[mu]
            if not (lo <= dd <= hi):
                return False
        return True
    def mask(par, width):
        m = np.zeros(V // 2)
        for lex in range(V):
            if sum(coords(dims, lex)) % 2 == par and in_region(lex, width):
                m[lex // 2] = 1
        return np.kron(np.ones(Ls), np.repeat(m, 12))
    M4oe = dense_of(lambda v: o.m4(v, 0), o.cb_shape())
    M4eo = dense_of(lambda v: o.m4(v, 1), o.cb_shape())
    n = M4oe.shape[0]
    M5i = dense_of(lambda v: o.apply5(o.matrix5(3), v), o.cb_shape())
    Pe, Po = np.diag(mask(0, pad)), np.diag(mask(1, pad))
    Be = np.diag(mask(0, 0))
    K = M5i @ Pe @ M4eo @ Po @ M5i @ Po @ M4oe @ Pe
    Dp = np.eye(n) - K
    return Be @ Dp.conj().T @ Dp @ Be


def test_local_operator_snake_terms(orc):
    dims, Ls, sub = (8, 2, 2, 2), 2, (2, 2, 2, 2)
    o, _ = make(orc, dims, Ls, eps=0.7)
    bid, nb = o.block_ids(sub)
    assert nb == 4
    blk = 1  # block at x = 2..3
    A_loc = dense_of(lambda v: o.local_DdagD(v, sub, block=blk), o.cb_shape())
    origin = (2, 0, 0, 0)
    A_pad2 = _padded_local(o, dims, Ls, sub, origin, 2)
    np.testing.assert_allclose(A_loc, A_pad2, atol=1e-12)
    # the sequentially truncated product (Dirichlet on every hop) is different
    A_trunc = _padded_local(o, dims, Ls, sub, origin, 0)
    assert np.abs(A_loc - A_trunc).max() > 1e-3
    # the oracle's truncated operator (vector form) is that dense product
    A_tr = dense_of(lambda v: o.local_DdagD_truncated(v, sub, block=blk), o.cb_shape())
    np.testing.assert_allclose(A_tr, A_trunc, atol=1e-12)
    # its even block mask agrees with block_ids
    np.testing.assert_array_equal(o.block_mask(sub, blk, 0) > 0, bid == blk)
    # and a pad of one is not enough to capture every snake
    A_pad1 = _padded_local(o, dims, Ls, sub, origin, 1)
    assert np.abs(A_loc - A_pad1).max() > 1e-4
    # the block-diagonal sum of all blocks is the oracle's (+)_s A_s
    x = rnd(o.cb_shape(), 3)
    tot = sum(o.local_DdagD(x, sub, block=k) for k in range(nb))
    np.testing.assert_allclose(tot, o.local_DdagD(x, sub), atol=1e-12)


def test_local_operator_unpartitioned_is_global(orc):
    dims, Ls = (4, 2, 2, 2), 3
    o, _ = make(orc, dims, Ls)
    x = rnd(o.cb_shape(), 5)
    np.testing.assert_allclose(o.local_DdagD(x, dims), o.DdagD(x), atol=1e-13)


# ------------------------------------------------------------ solvers


def _textbook_pcg(A, b, Minv, tol, maxit, pr=False):
    x = np.zeros_like(b); r = b.copy(); z = Minv(r); p = z.copy()
    rz = np.vdot(r, z).real; hist = [np.linalg.norm(r) / np.linalg.norm(b)]
    for k in range(maxit):
        Ap = A @ p; a = rz / np.vdot(p, Ap).real
        x = x + a * p; rn = r - a * Ap; zn = Minv(rn)
        beta = (np.vdot(zn, rn - r).real if pr else np.vdot(zn, rn).real) / rz
        rz = np.vdot(zn, rn).real
        p = zn + beta * p; r = rn; z = zn
        hist.append(np.linalg.norm(r) / np.linalg.norm(b))
        if hist[-1] < tol:
            break
    return x, np.array(hist)


def test_true_residual_is_the_relative_residual(orc):
    """The residual every GPU solve test is decided by: ||b - D^+D x|| / ||b|| in
    FP64, against the dense matrix (assembled column by column) and numpy's
    norms; 1 at x = 0, rounding level at the dense LU solution."""
    o, _ = make(orc, (2, 2, 2, 2), 4, mass=0.1)
    A = dense_of(o.DdagD, o.cb_shape())
    b, x = rnd(o.cb_shape(), 21), rnd(o.cb_shape(), 22)
    assert abs(o.true_residual(np.zeros_like(b), b) - 1.0) < 1e-15
    want = np.linalg.norm(b.reshape(-1) - A @ x.reshape(-1)) / np.linalg.norm(b)
    assert abs(o.true_residual(x, b) - want) <= 1e-12 * want
    xs = np.linalg.solve(A, b.reshape(-1)).reshape(b.shape)
    assert o.true_residual(xs, b) < 1e-12
    assert abs(o.true_residual(xs + 1e-3 * x, b) - 1e-3 * np.linalg.norm(A @ x.reshape(-1))
               / np.linalg.norm(b)) < 1e-9


def test_cg_matches_textbook_and_converges(orc):
    dims, Ls = (2, 2, 2, 4), 4
    o, _ = make(orc, dims, Ls, mass=0.05)
    A = dense_of(o.DdagD, o.cb_shape())
    b = rnd(o.cb_shape(), 6)
    res = o.pcg(b, tol=1e-10, maxiter=500, history=True)
    x_tb, h_tb = _textbook_pcg(A, b.reshape(-1), lambda r: r, 1e-10, 500)
    assert res["converged"] and res["true_res"] < 1e-10
    # identical iterates until rounding (different summation order) decorrelates them
    np.testing.assert_allclose(res["history"][:25], h_tb[:25], rtol=1e-7)
    assert abs(res["iters"] - (len(h_tb) - 1)) <= 0.1 * res["iters"]
    np.testing.assert_allclose(res["x"].reshape(-1), np.linalg.solve(A, b.reshape(-1)), atol=1e-8)


def test_mspcg_exact_block_inverse_is_block_jacobi_pcg(orc):
    """With enough inner iterations the inner CG is an exact block solve, so
    MSPCG equals textbook block-Jacobi PCG."""
    dims, Ls, sub = (8, 2, 2, 2), 2, (4, 2, 2, 2)
    o, _ = make(orc, dims, Ls, mass=0.1)
    A = dense_of(o.DdagD, o.cb_shape())
    b = rnd(o.cb_shape(), 7)
    bid, nb = o.block_ids(sub)
    sel = [np.kron(np.ones(Ls), np.repeat(bid == k, 12)).astype(bool) for k in range(nb)]
    def Minv(r):
        z = np.zeros_like(r)
        for m in sel:
            z[m] = np.linalg.solve(A[np.ix_(m, m)], r[m])
        return z
    x_tb, h_tb = _textbook_pcg(A, b.reshape(-1), Minv, 1e-10, 200, pr=True)
    res = o.pcg(b, precond=orc.PREC_MSPCG, beta=orc.BETA_PR, k=120, sub=sub, tol=1e-10,
                maxiter=200, history=True)
    assert res["iters"] == len(h_tb) - 1
    np.testing.assert_allclose(res["history"][:6], h_tb[:6], rtol=1e-5)


@pytest.mark.parametrize("k", [1, 2, 3, 5])
def test_preconditioner_is_k_steps_of_block_cg(orc, k):
    """z = M^-1 r of Sec. 2.4/2.5: on every block, exactly k CG iterations from
    a zero guess on the block's principal submatrix of D^+D.  k steps of CG
    from zero give the unique A-norm minimiser over the k-dimensional Krylov
    space, so a textbook CG on the dense blocks fixes the result."""
    dims, Ls, sub = (8, 2, 2, 2), 2, (4, 2, 2, 2)
    o, _ = make(orc, dims, Ls, mass=0.1)
    A = dense_of(o.DdagD, o.cb_shape())
    r = rnd(o.cb_shape(), 9)
    bid, nb = o.block_ids(sub)
    z_tb = np.zeros(r.size, dtype=np.complex128)
    rv = r.reshape(-1)
    for blk in range(nb):
        m = np.kron(np.ones(Ls), np.repeat(bid == blk, 12)).astype(bool)
        As, bs = A[np.ix_(m, m)], rv[m]
        x, res, p = np.zeros_like(bs), bs.copy(), bs.copy()
        rr = np.vdot(res, res).real
        for _ in range(k):
            Ap = As @ p
            al = rr / np.vdot(p, Ap).real
            x, res = x + al * p, res - al * Ap
            rr_new = np.vdot(res, res).real
            p, rr = res + (rr_new / rr) * p, rr_new
        z_tb[m] = x
    z = o.precond(r, orc.PREC_MSPCG, k=k, sub=sub)
    np.testing.assert_allclose(z.reshape(-1), z_tb, rtol=0, atol=1e-11 * np.abs(z_tb).max())
    if k < 5:  # not yet the exact block solve
        z_exact = np.zeros_like(z_tb)
        for blk in range(nb):
            m = np.kron(np.ones(Ls), np.repeat(bid == blk, 12)).astype(bool)
            z_exact[m] = np.linalg.solve(A[np.ix_(m, m)], rv[m])
        assert np.linalg.norm(z_tb - z_exact) > 1e-6 * np.linalg.norm(z_exact)


def test_identity_preconditioner_reproduces_cg(orc):
    """Reduced-Ls form with Ls_hat = Ls, T = 1 and mu = 0 is the plain MSPCG
    preconditioner; with the identity (no preconditioner) PCG+FR is CG."""
    dims, Ls, sub = (4, 2, 2, 4), 4, (4, 2, 2, 2)
    o, _ = make(orc, dims, Ls)
    r = rnd(o.cb_shape(), 8)
    T = np.eye(4 * Ls)
    z1 = o.precond(r, orc.PREC_MSPCG, k=4, sub=sub)
    z2 = o.precond(r, orc.PREC_REDUCED, k=4, sub=sub, Ls_hat=Ls, T=T, mu=0.0)
    np.testing.assert_allclose(z1, z2, atol=1e-13)
    z3 = o.precond(r, orc.PREC_REDUCED, k=4, sub=sub, Ls_hat=Ls, T=T, mu=0.3)
    np.testing.assert_allclose(z3, z1 + 0.3 * r, atol=1e-13)


def test_reduced_preconditioner_composes_its_pinned_parts(orc):
    """Sec. 3.3: z = T^+ (k CG steps on Mhat) T r + mu r, with Mhat the local
    operator at Ls_hat; composed here from the separately pinned T map and the
    k-step block CG at Ls_hat, for a random complex T."""
    dims, Ls, Lsh, sub, k = (8, 2, 2, 2), 4, 2, (4, 2, 2, 2), 3
    o, _ = make(orc, dims, Ls, mass=0.1)
    oh = o.with_Ls(Lsh)
    rng = np.random.default_rng(12)
    T = rng.standard_normal((4 * Lsh, 4 * Ls)) + 1j * rng.standard_normal((4 * Lsh, 4 * Ls))
    r = rnd(o.cb_shape(), 13)
    want = o.T_apply(T, oh.precond(o.T_apply(T, r, Lsh), orc.PREC_MSPCG, k=k, sub=sub), Lsh,
                     dagger=True) + 0.4 * r
    got = o.precond(r, orc.PREC_REDUCED, k=k, sub=sub, Ls_hat=Lsh, T=T, mu=0.4)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12 * np.abs(want).max())


def test_reduced_ls_operator_hermitian(orc):
    """T^+ Mhat^-1 T is Hermitian and rank deficient for Ls_hat < Ls (Sec. 3.3)."""
    dims, Ls, Lsh, sub = (2, 2, 2, 2), 4, 2, (2, 2, 2, 2)
    o, _ = make(orc, dims, Ls)
    oh = o.with_Ls(Lsh)
    rng = np.random.default_rng(1)
    T = rng.standard_normal((4 * Lsh, 4 * Ls)) + 1j * rng.standard_normal((4 * Lsh, 4 * Ls))
    Ah = dense_of(oh.DdagD, oh.cb_shape())
    Ahi = np.linalg.inv(Ah)
    def op(v):
        vh = o.T_apply(T, v, Lsh)
        w = (Ahi @ vh.reshape(-1)).reshape(vh.shape)
        return o.T_apply(T, w, Lsh, dagger=True)
    Mred = dense_of(op, o.cb_shape())
    np.testing.assert_allclose(Mred, Mred.conj().T, atol=1e-10)
    ev = np.linalg.eigvalsh(Mred)
    assert (np.abs(ev) < 1e-9 * np.abs(ev).max()).sum() == Mred.shape[0] // 2
    # T adjoint application is the conjugate transpose
    x, y = rnd(o.cb_shape(), 2), rnd(oh.cb_shape(), 3)
    assert abs(np.vdot(y, o.T_apply(T, x, Lsh)) - np.vdot(o.T_apply(T, y, Lsh, True), x)) < 1e-10


def test_T_apply_selection_is_indexing(orc):
    """T indexed (s, spin) x (t, spin') (Sec. 3.3: T acts on spin x fifth
    dimension, trivially on colour and sites).  A T that picks slice sel[s]
    and spin perm[a] for output (s, a) must reduce to array indexing, and T^+
    to the matching scatter; a transposed or reordered (s, spin) index fails."""
    dims, Ls, Lsh = (2, 2, 2, 2), 6, 3
    o, _ = make(orc, dims, Ls)
    sel, perm = [4, 0, 2], [2, 0, 3, 1]
    T = np.zeros((4 * Lsh, 4 * Ls), dtype=np.complex128)
    for s in range(Lsh):
        for a in range(4):
            T[s * 4 + a, sel[s] * 4 + perm[a]] = 1.0
    x = rnd(o.cb_shape(), 5)
    y = o.T_apply(T, x, Lsh)
    np.testing.assert_array_equal(y, x[sel][:, :, perm, :])
    back = o.T_apply(T, y, Lsh, dagger=True)
    want = np.zeros_like(x)
    for s in range(Lsh):
        want[sel[s]][:, perm, :] = y[s]
    np.testing.assert_array_equal(back, want)
    # a complex phase per row is conjugated by the adjoint
    ph = np.exp(1j * np.arange(4 * Lsh))
    y2 = o.T_apply(ph[:, None] * T, x, Lsh)
    np.testing.assert_allclose(y2, y * ph.reshape(Lsh, 1, 4, 1), rtol=0, atol=1e-15)
    back2 = o.T_apply(ph[:, None] * T, y2, Lsh, dagger=True)
    np.testing.assert_allclose(back2, want, rtol=0, atol=1e-14)


def test_mspcg_reduces_outer_iterations(orc):
    """Qualitative (Sec. 2.5): with 6 inner iterations the outer count drops."""
    dims, Ls, sub = (8, 4, 4, 4), 4, (4, 4, 4, 4)
    o, _ = make(orc, dims, Ls, mass=0.02, eps=0.4, seed=3)
    b = rnd(o.cb_shape(), 12)
    cg = o.pcg(b, tol=1e-8, maxiter=2000)
    ms = o.pcg(b, precond=orc.PREC_MSPCG, beta=orc.BETA_PR, k=6, sub=sub, tol=1e-8, maxiter=2000)
    assert cg["converged"] and ms["converged"]
    assert ms["true_res"] < 1.5e-8
    assert ms["iters"] < cg["iters"] / 2


# ------------------------------------------------- reduced-Ls transform loss


def test_T_loss_gradient_matches_finite_differences(orc):
    """Sec. 3.3 loss: the analytic gradient G (d chi^2 = 2 Re <G, dT>) against
    central differences of chi^2 along random complex directions."""
    dims, Ls, Lh, sub = (8, 2, 2, 2), 4, 2, (4, 2, 2, 2)
    o, _ = make(orc, dims, Ls, eps=0.5, mass=0.1)
    rng = np.random.default_rng(7)
    vs = [rnd(o.cb_shape(), 11), rnd(o.cb_shape(), 12)]
    T = rng.standard_normal((4 * Lh, 4 * Ls)) + 1j * rng.standard_normal((4 * Lh, 4 * Ls))
    mu = 0.3
    chi2, G = o.T_loss(T, mu, vs, sub, Lh)
    assert chi2 > 0
    for seed in (1, 2):
        D = np.random.default_rng(seed).standard_normal(T.shape) + 1j * np.random.default_rng(seed + 9).standard_normal(T.shape)
        h = 1e-4
        cp, _ = o.T_loss(T + h * D, mu, vs, sub, Lh, grad=False)
        cm, _ = o.T_loss(T - h * D, mu, vs, sub, Lh, grad=False)
        fd = (cp - cm) / (2 * h)
        an = 2 * np.real(np.vdot(G, D))
        assert abs(fd - an) <= 1e-6 * abs(an), (fd, an)


def test_T_loss_vanishes_at_identity(orc):
    """With Ls_hat = Ls, T = 1 and mu = 0 the reduced preconditioner is M^-1
    itself: chi^2 = 0 and the gradient vanishes."""
    dims, Ls, sub = (8, 2, 2, 2), 4, (4, 2, 2, 2)
    o, _ = make(orc, dims, Ls, eps=0.5, mass=0.1)
    vs = [rnd(o.cb_shape(), 21)]
    chi2, G = o.T_loss(np.eye(4 * Ls, dtype=np.complex128), 0.0, vs, sub, Ls)
    vv = sum(np.vdot(v, v).real for v in vs)
    assert chi2 <= 1e-20 * vv
    assert np.abs(G).max() <= 1e-9 * np.sqrt(vv)
