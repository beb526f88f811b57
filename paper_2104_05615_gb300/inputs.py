"""Seeded synthetic inputs shared by the CUDA path, the oracle tests and the bench.

This module draws random numbers and builds the synthetic gauge field and
sources; it holds none of the solver's arithmetic (no Dirac operator, no
fifth-dimension matrices, no Krylov step).

Random numbers: a counter-based SplitMix64 (Steele, Lea, Flood, "Fast
splittable pseudorandom number generators", OOPSLA 2014): the i-th draw of
stream (seed, stream_id) is mix64(key + (i+1)*GOLDEN) with
key = mix64(seed ^ (stream_id << 32) ^ GOLDEN).  Uniforms use the top 53
bits; normals use the Box-Muller transform in FP64.

Gauge field (Sec. 2.2 describes links as SU(3) matrices between 4D sites):
each link is U = exp(i*eps*H) with H = sum_a w_a lambda_a / 2, w_a ~ N(0,1)
i.i.d. and lambda_a the Gell-Mann matrices, exponentiated through the
eigendecomposition of the Hermitian H.  eps = 0 gives the unit (free) field.

Layouts (the canonical layouts of the C ABI):
  gauge   [V][4][3][3] complex128, site index lex = x + Lx*(y + Ly*(z + Lz*t))
  even/odd 5D spinor [Ls][V/2][4][3] complex128, site index lex//2 over the
          sites of one parity (x+y+z+t) mod 2.
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix64(z: np.ndarray) -> np.ndarray:
    z = z.copy()
    z ^= z >> np.uint64(30)
    z *= _M1
    z ^= z >> np.uint64(27)
    z *= _M2
    z ^= z >> np.uint64(31)
    return z


def splitmix64(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """n uint64 draws of stream (seed, stream), starting at counter `offset`."""
    with np.errstate(over="ignore"):
        key = _mix64(np.array([(seed ^ (stream << 32)) & 0xFFFFFFFFFFFFFFFF],
                              dtype=np.uint64) ^ _GOLDEN)[0]
        ctr = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        return _mix64(key + ctr * _GOLDEN)


def uniform(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """Uniform doubles in (0, 1)."""
    u = splitmix64(seed, stream, n, offset) >> np.uint64(11)
    return (u.astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)


def normal(seed: int, stream: int, n: int) -> np.ndarray:
    """n i.i.d. N(0,1) doubles by Box-Muller (pairs of uniforms)."""
    m = (n + 1) // 2
    out = np.empty(2 * m, dtype=np.float64)
    chunk = 1 << 24
    for lo in range(0, m, chunk):
        hi = min(m, lo + chunk)
        u = uniform(seed, stream, 2 * (hi - lo), 2 * lo)
        u1, u2 = u[0::2], u[1::2]
        r = np.sqrt(-2.0 * np.log(u1))
        th = 2.0 * np.pi * u2
        out[2 * lo:2 * hi:2] = r * np.cos(th)
        out[2 * lo + 1:2 * hi:2] = r * np.sin(th)
    return out[:n]


def gell_mann() -> np.ndarray:
    """The eight Gell-Mann matrices, tr(l_a l_b) = 2 delta_ab."""
    l = np.zeros((8, 3, 3), dtype=np.complex128)
    l[0, 0, 1] = l[0, 1, 0] = 1
    l[1, 0, 1], l[1, 1, 0] = -1j, 1j
    l[2, 0, 0], l[2, 1, 1] = 1, -1
    l[3, 0, 2] = l[3, 2, 0] = 1
    l[4, 0, 2], l[4, 2, 0] = -1j, 1j
    l[5, 1, 2] = l[5, 2, 1] = 1
    l[6, 1, 2], l[6, 2, 1] = -1j, 1j
    l[7] = np.diag([1, 1, -2]) / np.sqrt(3.0)
    return l


def su3_exp_field(n: int, eps: float, seed: int, stream: int = 0) -> np.ndarray:
    """n matrices exp(i*eps*H), H Gaussian traceless Hermitian; shape (n,3,3)."""
    w = normal(seed, stream, 8 * n).reshape(n, 8)
    lam = gell_mann()
    out = np.empty((n, 3, 3), dtype=np.complex128)
    chunk = 1 << 20
    for lo in range(0, n, chunk):
        hi = min(n, lo + chunk)
        H = np.einsum("na,aij->nij", w[lo:hi], lam) * 0.5
        h, V = np.linalg.eigh(H)
        ph = np.exp(1j * eps * h)
        out[lo:hi] = np.einsum("nij,nj,nkj->nik", V, ph, V.conj())
    return out


def gauge_field(dims, eps: float, seed: int) -> np.ndarray:
    """Seeded SU(3) gauge field, shape (V, 4, 3, 3), link (site, mu)."""
    V = int(np.prod(dims))
    return su3_exp_field(V * 4, eps, seed).reshape(V, 4, 3, 3)


def random_su3(n: int, seed: int) -> np.ndarray:
    """Random SU(3) matrices (eps = 1 exponentials) for gauge-transform tests."""
    return su3_exp_field(n, 1.0, seed, stream=7)


def gaussian_spinor_cb(dims, Ls: int, seed: int, stream: int = 0) -> np.ndarray:
    """Gaussian even/odd 5D spinor, complex128 of shape (Ls, V/2, 4, 3)."""
    Vh = int(np.prod(dims)) // 2
    n = Ls * Vh * 12
    re_im = normal(seed, stream, 2 * n)
    out = re_im.view(np.complex128)
    return out.reshape(Ls, Vh, 4, 3)


def gaussian_spinor_full(dims, Ls: int, seed: int, stream: int = 0) -> np.ndarray:
    """Gaussian full-lattice 5D spinor, complex128 of shape (Ls, V, 4, 3)."""
    V = int(np.prod(dims))
    re_im = normal(seed, stream, 2 * Ls * V * 12)
    return re_im.view(np.complex128).reshape(Ls, V, 4, 3)


def plaquette(U: np.ndarray, dims) -> float:
    """Average plaquette Re tr(U U U^+ U^+)/3, a fingerprint of the field."""
    Lx, Ly, Lz, Lt = dims
    G = U.reshape(Lt, Lz, Ly, Lx, 4, 3, 3)
    axis = {0: 3, 1: 2, 2: 1, 3: 0}
    tot = 0.0
    for mu in range(4):
        for nu in range(mu + 1, 4):
            Um = G[..., mu, :, :]
            Un = G[..., nu, :, :]
            Un_xmu = np.roll(Un, -1, axis=axis[mu])
            Um_xnu = np.roll(Um, -1, axis=axis[nu])
            P = Um @ Un_xmu @ np.conj(np.swapaxes(Um_xnu, -1, -2)) \
                @ np.conj(np.swapaxes(Un, -1, -2))
            tot += np.mean(np.real(np.trace(P, axis1=-2, axis2=-1))) / 3.0
    return tot / 6.0


# Workload recipes.  b, c, M5 are common; eps is the gauge "temperature";
# seeds for gauge / source.  These reproduce the shapes of the paper's
# workloads (Ls = 12/16, 8^4 and 16^4 blocks, k = 6 inner iterations).
CONFIGS = {
    "C1": dict(dims=(4, 4, 4, 4), Ls=8, b=1.5, c=0.5, M5=1.8, mass=0.01,
               eps=0.3, gauge_seed=101, src_seed=201, tol=1e-10,
               solver="cg", outer_prec="f64", sub=(4, 4, 4, 4)),
    "C2": dict(dims=(8, 8, 8, 8), Ls=12, b=1.5, c=0.5, M5=1.8, mass=0.005,
               eps=0.5, gauge_seed=102, src_seed=202, tol=1e-10,
               solver="cg", outer_prec="f32", sub=(8, 8, 8, 8)),
    "C3": dict(dims=(16, 16, 16, 32), Ls=12, b=1.5, c=0.5, M5=1.8, mass=0.002,
               eps=0.6, gauge_seed=103, src_seed=203, tol=1e-10,
               solver="mspcg", outer_prec="f32", inner_prec="f16",
               inner_iters=6, sub=(8, 8, 8, 8)),
    "C4": dict(dims=(32, 32, 32, 64), Ls=16, b=1.5, c=0.5, M5=1.8, mass=0.001,
               eps=0.7, gauge_seed=104, src_seed=204, tol=1e-10,
               solver="mspcg", outer_prec="f32", inner_prec="bf16",
               inner_iters=6, sub=(16, 16, 16, 16), Ls_hat=8, mu=0.85),
}


def c5_systems():
    """The 48 independent systems of the batched workload: 16 each of 8^4,
    8^3x16 and 12^4, Ls=12, 4^4 blocks, mass ~ U[0.002, 0.02] (seed 305)."""
    masses = 0.002 + 0.018 * uniform(305, 0, 48)
    shapes = [(8, 8, 8, 8)] * 16 + [(8, 8, 8, 16)] * 16 + [(12, 12, 12, 12)] * 16
    out = []
    for i, d in enumerate(shapes):
        out.append(dict(dims=d, Ls=12, b=1.5, c=0.5, M5=1.8, mass=float(masses[i]),
                        eps=0.5, gauge_seed=1000 + i, src_seed=2000 + i, tol=1e-9,
                        sub=(4, 4, 4, 4), inner_iters=6))
    return out
