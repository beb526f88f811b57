"""Independent dense constructions used to pin the oracle (test code only).

Everything here is assembled in numpy from textbook definitions, with its own
explicit gamma matrices, so that a mistake in the oracle's gamma table, hop
assembly, fifth-dimension matrices or even/odd bookkeeping shows up as a
mismatch.
"""
import numpy as np

# Chiral (DeGrand-Rossi) basis written out entry by entry.
G = np.array([
    [[0, 0, 0, 1j], [0, 0, 1j, 0], [0, -1j, 0, 0], [-1j, 0, 0, 0]],
    [[0, 0, 0, 1], [0, 0, -1, 0], [0, -1, 0, 0], [1, 0, 0, 0]],
    [[0, 0, 1j, 0], [0, 0, 0, -1j], [-1j, 0, 0, 0], [0, 1j, 0, 0]],
    [[0, 0, 1, 0], [0, 0, 0, 1], [1, 0, 0, 0], [0, 1, 0, 0]],
], dtype=np.complex128)
G5 = np.diag([-1, -1, 1, 1]).astype(np.complex128)
PPLUS = (np.eye(4) + G5) / 2
PMINUS = (np.eye(4) - G5) / 2


def coords(dims, lex):
    Lx, Ly, Lz, Lt = dims
    return [lex % Lx, (lex // Lx) % Ly, (lex // (Lx * Ly)) % Lz, lex // (Lx * Ly * Lz)]


def lexi(dims, x):
    Lx, Ly, Lz, Lt = dims
    return x[0] + Lx * (x[1] + Ly * (x[2] + Lz * x[3]))


def parity(dims, lex):
    return sum(coords(dims, lex)) & 1


def wilson_hop_dense(U, dims):
    """Dense 4D D^w, index lex*12 + spin*3 + colour."""
    V = int(np.prod(dims))
    D = np.zeros((12 * V, 12 * V), dtype=np.complex128)
    I4 = np.eye(4)
    for lex in range(V):
        x = coords(dims, lex)
        for mu in range(4):
            xp = list(x); xp[mu] = (x[mu] + 1) % dims[mu]
            xm = list(x); xm[mu] = (x[mu] - 1) % dims[mu]
            yp, ym = lexi(dims, xp), lexi(dims, xm)
            D[12 * lex:12 * lex + 12, 12 * yp:12 * yp + 12] += np.kron(I4 - G[mu], U[lex, mu])
            D[12 * lex:12 * lex + 12, 12 * ym:12 * ym + 12] += np.kron(I4 + G[mu], U[ym, mu].conj().T)
    return D


def chiral_shift_5d(Ls, V, mass):
    """P acting on (s, site, spin, colour): P_- psi_{s+1} + P_+ psi_{s-1}, wraps -mass."""
    Eup = np.zeros((Ls, Ls)); Edn = np.zeros((Ls, Ls))
    for s in range(Ls):
        if s + 1 < Ls: Eup[s, s + 1] = 1
        else: Eup[s, 0] = -mass
        if s - 1 >= 0: Edn[s, s - 1] = 1
        else: Edn[s, Ls - 1] = -mass
    site = np.eye(V)
    return (np.kron(Eup, np.kron(site, np.kron(PMINUS, np.eye(3)))) +
            np.kron(Edn, np.kron(site, np.kron(PPLUS, np.eye(3)))))


def mobius_d5_textbook(U, dims, Ls, b, c, M5, mass):
    """D5 = (b D_W + 1) - (1 - c D_W) P with D_W = (4 - M5) - D^w / 2."""
    V = int(np.prod(dims))
    Dw = wilson_hop_dense(U, dims)
    DW = (4.0 - M5) * np.eye(12 * V) - 0.5 * Dw
    Dp = b * DW + np.eye(12 * V)
    Dm = np.eye(12 * V) - c * DW
    P = chiral_shift_5d(Ls, V, mass)
    I5 = np.eye(Ls)
    return np.kron(I5, Dp) - np.kron(I5, Dm) @ P


def dense_of(fn, shape_in):
    """Dense matrix of a linear map by applying it to unit vectors."""
    n = int(np.prod(shape_in))
    cols = []
    for j in range(n):
        e = np.zeros(n, dtype=np.complex128)
        e[j] = 1.0
        cols.append(np.asarray(fn(e.reshape(shape_in))).reshape(-1))
    return np.stack(cols, axis=1)


def parity_index(dims, Ls, par):
    """Indices of the full 5D vector (s, lex, 12) that belong to an even/odd
    field (s, lex//2, 12) of parity par, in the even/odd field's order."""
    V = int(np.prod(dims))
    lex_of = np.zeros(V // 2, dtype=np.int64)
    for lex in range(V):
        if parity(dims, lex) == par:
            lex_of[lex // 2] = lex
    idx = []
    for s in range(Ls):
        for h in range(V // 2):
            base = (s * V + lex_of[h]) * 12
            idx.extend(range(base, base + 12))
    return np.array(idx)


def gauge_transform(U, g, dims):
    """U'_mu(x) = g(x) U_mu(x) g(x+mu)^+."""
    V = int(np.prod(dims))
    Up = np.empty_like(U)
    for lex in range(V):
        x = coords(dims, lex)
        for mu in range(4):
            xp = list(x); xp[mu] = (x[mu] + 1) % dims[mu]
            Up[lex, mu] = g[lex] @ U[lex, mu] @ g[lexi(dims, xp)].conj().T
    return Up
