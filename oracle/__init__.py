"""ctypes wrapper of the FP64 CPU oracle (oracle/dwf_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check and by the
bench's CPU-baseline / reference leg.  The CUDA library never imports it.

Arrays are numpy complex128 in the canonical layouts documented in
dwf_oracle.h: even/odd fields (Ls, V/2, 4, 3), full fields (Ls, V, 4, 3),
gauge (V, 4, 3, 3).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dwf_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liborc.so")
_lock = threading.Lock()
_lib = None

P, M5OP, MPHI, M5INV = 0, 1, 2, 3
PREC_NONE, PREC_MSPCG, PREC_REDUCED = 0, 1, 2
BETA_FR, BETA_PR = 0, 1


def build(force: bool = False) -> str:
    """Compile the oracle with the host C compiler (gcc, OpenMP)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    stale = (not os.path.exists(_LIB) or
             os.path.getmtime(_LIB) < max(os.path.getmtime(_SRC),
                                          os.path.getmtime(os.path.join(_HERE, "dwf_oracle.h"))))
    if force or stale:
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class Params(C.Structure):
    _fields_ = [("L", C.c_int * 4), ("Ls", C.c_int), ("b", C.c_double), ("c", C.c_double),
                ("M5", C.c_double), ("mass", C.c_double), ("antiperiodic_t", C.c_int)]


class Solver(C.Structure):
    _fields_ = [("precond", C.c_int), ("beta", C.c_int), ("inner_iters", C.c_int),
                ("sub", C.c_int * 4), ("tol", C.c_double), ("maxiter", C.c_int),
                ("Ls_hat", C.c_int), ("T", C.c_void_p), ("mu", C.c_double)]


class Result(C.Structure):
    _fields_ = [("iters", C.c_int), ("true_res", C.c_double), ("converged", C.c_int)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            _lib.orc_true_residual.restype = C.c_double
            _lib.orc_block_ids.restype = C.c_long
    return _lib


def _ptr(a: np.ndarray):
    assert a.flags.c_contiguous
    return a.ctypes.data_as(C.c_void_p)


def _c(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.complex128)


def num_threads() -> int:
    return lib().orc_num_threads()


class Oracle:
    """The operators of one lattice (params + gauge field)."""

    def __init__(self, dims, Ls, b, c, M5, mass, gauge, antiperiodic_t=0):
        self.dims = tuple(int(d) for d in dims)
        self.Ls = int(Ls)
        self.V = int(np.prod(self.dims))
        self.Vh = self.V // 2
        self.p = Params((C.c_int * 4)(*self.dims), self.Ls, b, c, M5, mass, antiperiodic_t)
        self.gauge = _c(gauge).reshape(self.V, 4, 3, 3)
        self.b, self.c, self.M5, self.mass = b, c, M5, mass
        self.antiperiodic_t = antiperiodic_t

    def with_Ls(self, Ls):
        return Oracle(self.dims, Ls, self.b, self.c, self.M5, self.mass, self.gauge,
                      self.antiperiodic_t)

    # -- shapes
    def cb_shape(self, Ls=None):
        return (Ls or self.Ls, self.Vh, 4, 3)

    def full_shape(self):
        return (self.Ls, self.V, 4, 3)

    # -- operators
    def hop(self, x, dagger=False):
        x = _c(x).reshape(self.full_shape())
        out = np.empty_like(x)
        lib().orc_hop(C.byref(self.p), _ptr(self.gauge), _ptr(x), _ptr(out), int(dagger))
        return out

    def matrix5(self, which, dagger=False):
        n = 4 * self.Ls
        M = np.empty((n, n), dtype=np.complex128)
        lib().orc_5d_matrix(C.byref(self.p), which, int(dagger), _ptr(M))
        return M

    def m5inv_closed(self, chirality):
        M = np.empty((self.Ls, self.Ls), dtype=np.float64)
        lib().orc_m5inv_closed(C.byref(self.p), int(chirality), _ptr(M))
        return M

    def apply5(self, M, x):
        x = _c(x)
        nsite = x.shape[1]
        out = np.empty_like(x)
        lib().orc_apply_5d(C.byref(self.p), _ptr(_c(M)), _ptr(x), _ptr(out), C.c_long(nsite))
        return out

    def D5(self, x):
        x = _c(x).reshape(self.full_shape())
        out = np.empty_like(x)
        lib().orc_D5(C.byref(self.p), _ptr(self.gauge), _ptr(x), _ptr(out))
        return out

    def m4(self, x, in_par, dagger=False):
        x = _c(x).reshape(self.cb_shape())
        out = np.empty_like(x)
        lib().orc_m4(C.byref(self.p), _ptr(self.gauge), _ptr(x), int(in_par), _ptr(out), int(dagger))
        return out

    def D(self, x, dagger=False):
        x = _c(x).reshape(self.cb_shape())
        out = np.empty_like(x)
        lib().orc_Deo(C.byref(self.p), _ptr(self.gauge), _ptr(x), _ptr(out), int(dagger))
        return out

    def DdagD(self, x):
        x = _c(x).reshape(self.cb_shape())
        out = np.empty_like(x)
        lib().orc_DdagD(C.byref(self.p), _ptr(self.gauge), _ptr(x), _ptr(out))
        return out

    def phihat(self, phi_full):
        phi = _c(phi_full).reshape(self.full_shape())
        out = np.empty(self.cb_shape(), dtype=np.complex128)
        lib().orc_phihat(C.byref(self.p), _ptr(self.gauge), _ptr(phi), _ptr(out))
        return out

    def reconstruct_odd(self, psi_e, phi_full):
        psi = _c(psi_e).reshape(self.cb_shape())
        phi = _c(phi_full).reshape(self.full_shape())
        out = np.empty(self.cb_shape(), dtype=np.complex128)
        lib().orc_reconstruct_odd(C.byref(self.p), _ptr(self.gauge), _ptr(psi), _ptr(phi), _ptr(out))
        return out

    def block_ids(self, sub):
        bid = np.empty(self.Vh, dtype=np.int32)
        n = lib().orc_block_ids(C.byref(self.p), _ptr(np.ascontiguousarray(sub, dtype=np.int32)),
                                _ptr(bid))
        return bid, int(n)

    def local_DdagD(self, x, sub, block=None):
        x = _c(x).reshape(self.cb_shape())
        out = np.empty_like(x)
        s = np.ascontiguousarray(sub, dtype=np.int32)
        if block is None:
            lib().orc_local_DdagD(C.byref(self.p), _ptr(self.gauge), _ptr(s), _ptr(x), _ptr(out))
        else:
            lib().orc_local_DdagD_block(C.byref(self.p), _ptr(self.gauge), _ptr(s),
                                        C.c_long(block), _ptr(x), _ptr(out))
        return out

    def block_mask(self, sub, block, par):
        """1 on the sites of checkerboard `par` (cb index lex // 2) that lie in
        block `block` (numbered as block_ids), else 0; shape (Vh,)."""
        nb = [self.dims[mu] // sub[mu] for mu in range(4)]
        m = np.zeros(self.Vh)
        for lex in range(self.V):
            x, t = [], lex
            for mu in range(4):
                x.append(t % self.dims[mu])
                t //= self.dims[mu]
            if sum(x) % 2 != par:
                continue
            b = x[0] // sub[0] + nb[0] * (x[1] // sub[1] + nb[1] * (x[2] // sub[2] + nb[2] * (x[3] // sub[3])))
            if b == block:
                m[lex // 2] = 1.0
        return m

    def local_DdagD_truncated(self, x, sub, block=None):
        """The left side of Eq. (eq:diri): D^+D with Dirichlet walls at the
        block boundary on each of its four hops (Sec. 2.3; the snake terms that
        leave the block and come back are dropped), on the block's even sites:
        P_e D_t^+ D_t P_e with D_t = 1 - M5^-1 P_e M4_eo P_o M5^-1 P_o M4_oe P_e.
        block None: the sum over all blocks."""
        x = _c(x).reshape(self.cb_shape())
        if block is None:
            nblk = int(np.prod([self.dims[mu] // sub[mu] for mu in range(4)]))
            return sum(self.local_DdagD_truncated(x, sub, b) for b in range(nblk))
        Pe = self.block_mask(sub, block, 0)[None, :, None, None]
        Po = self.block_mask(sub, block, 1)[None, :, None, None]
        Mi = self.matrix5(M5INV)
        Mid = Mi.conj().T

        def Dt(v):
            k = self.m4(Pe * v, 0)                     # M4_oe: even -> odd
            k = self.apply5(Mi, Po * k)
            k = self.m4(Po * k, 1)                     # M4_eo: odd -> even
            return v - self.apply5(Mi, Pe * k)

        def Dt_dag(v):
            k = Pe * self.apply5(Mid, v)
            k = Po * self.m4(k, 0, dagger=True)        # M4_eo^+: even -> odd
            k = Po * self.apply5(Mid, k)
            return v - Pe * self.m4(k, 1, dagger=True)  # M4_oe^+: odd -> even

        return Pe * Dt_dag(Dt(Pe * x))

    def reduced_local_inverse(self, r_hat, sub, Ls_hat, tol=1e-13, maxiter=5000):
        """Mhat^-1 r_hat for Mhat = (+)_s A_s at the reduced extent Ls_hat (same
        b, c, M5, mass): plain CG to a relative residual tol, i.e. the exact
        inverse the transform training of Sec. 3.3 differentiates through."""
        o = self.with_Ls(Ls_hat)
        b = _c(r_hat).reshape(o.cb_shape())
        x = np.zeros_like(b)
        r = b.copy()
        p = r.copy()
        rr = np.vdot(r, r).real
        bb = rr
        for _ in range(maxiter):
            if rr <= tol * tol * bb:
                break
            Ap = o.local_DdagD(p, sub)
            al = rr / np.vdot(p, Ap).real
            x += al * p
            r -= al * Ap
            rr_new = np.vdot(r, r).real
            p = r + (rr_new / rr) * p
            rr = rr_new
        return x

    @staticmethod
    def outer_contract(a, b):
        """sum over sites and colours of a b^+: rows s*4 + spin of a (La slices),
        columns t*4 + spin of b (Lb slices)."""
        La, Lb = a.shape[0], b.shape[0]
        return np.einsum("sxmc,txnc->smtn", a, np.conj(b)).reshape(4 * La, 4 * Lb)

    def T_loss(self, T, mu, vs, sub, Ls_hat, grad=True):
        """Sec. 3.3: chi^2(T) = sum_i |M (T^+ Mhat^-1 T + mu) v_i - v_i|^2, M the
        local operator (+)_s A_s at Ls, Mhat the one at Ls_hat.  With
        w = Mhat^-1 T v, e = M (T^+ w + mu v) - v, g = M e, u = Mhat^-1 T g,
        d chi^2 = 2 Re <G, dT>_F with G = sum_i (w_i g_i^+ + u_i v_i^+) (outer
        products contracted over sites and colours).  Returns (chi^2, G)."""
        chi2, G = 0.0, np.zeros_like(np.asarray(T, dtype=np.complex128))
        for v in vs:
            v = _c(v).reshape(self.cb_shape())
            w = self.reduced_local_inverse(self.T_apply(T, v, Ls_hat), sub, Ls_hat)
            e = self.local_DdagD(self.T_apply(T, w, Ls_hat, dagger=True) + mu * v, sub) - v
            chi2 += np.vdot(e, e).real
            if grad:
                g = self.local_DdagD(e, sub)
                u = self.reduced_local_inverse(self.T_apply(T, g, Ls_hat), sub, Ls_hat)
                G += self.outer_contract(w, g) + self.outer_contract(u, v)
        return chi2, G

    def T_apply(self, T, x, Ls_hat, dagger=False):
        x = _c(x)
        nsite = x.shape[1]
        Lout = self.Ls if dagger else Ls_hat
        out = np.empty((Lout, nsite, 4, 3), dtype=np.complex128)
        lib().orc_T_apply(_ptr(_c(T)), int(Ls_hat), int(self.Ls), C.c_long(nsite), _ptr(x),
                          _ptr(out), int(dagger))
        return out

    def true_residual(self, x, b):
        return lib().orc_true_residual(C.byref(self.p), _ptr(self.gauge),
                                       _ptr(_c(x).reshape(self.cb_shape())),
                                       _ptr(_c(b).reshape(self.cb_shape())))

    def _solver(self, precond, beta, k, sub, tol, maxiter, Ls_hat=0, T=None, mu=0.0):
        sv = Solver()
        sv.precond, sv.beta, sv.inner_iters = precond, beta, k
        sv.sub = (C.c_int * 4)(*(sub or self.dims))
        sv.tol, sv.maxiter = tol, maxiter
        sv.Ls_hat = Ls_hat
        self._T_keep = None if T is None else _c(T)
        sv.T = None if T is None else self._T_keep.ctypes.data
        sv.mu = mu
        return sv

    def precond(self, r, precond=PREC_MSPCG, k=6, sub=None, Ls_hat=0, T=None, mu=0.0):
        sv = self._solver(precond, BETA_PR, k, sub, 0.0, 0, Ls_hat, T, mu)
        r = _c(r).reshape(self.cb_shape())
        z = np.empty_like(r)
        lib().orc_precond(C.byref(self.p), _ptr(self.gauge), C.byref(sv), _ptr(r), _ptr(z))
        return z

    def pcg(self, b, x0=None, precond=PREC_NONE, beta=BETA_FR, k=6, sub=None, tol=1e-10,
            maxiter=10000, Ls_hat=0, T=None, mu=0.0, history=False):
        sv = self._solver(precond, beta, k, sub, tol, maxiter, Ls_hat, T, mu)
        b = _c(b).reshape(self.cb_shape())
        x = np.zeros_like(b) if x0 is None else _c(x0).reshape(self.cb_shape()).copy()
        res = Result()
        hist = np.zeros(maxiter + 1) if history else None
        lib().orc_pcg(C.byref(self.p), _ptr(self.gauge), C.byref(sv), _ptr(x), _ptr(b),
                      C.byref(res), None if hist is None else _ptr(hist))
        out = dict(x=x, iters=res.iters, true_res=res.true_res, converged=bool(res.converged))
        if history:
            out["history"] = hist[:res.iters + 1]
        return out


def gamma(mu: int) -> np.ndarray:
    g = np.empty((4, 4), dtype=np.complex128)
    lib().orc_gamma(int(mu), _ptr(g))
    return g


def from_config(cfg, gauge, Ls=None) -> Oracle:
    return Oracle(cfg["dims"], Ls or cfg["Ls"], cfg["b"], cfg["c"], cfg["M5"], cfg["mass"], gauge)
