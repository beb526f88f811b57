"""Training the reduced-Ls transform T (Sec. 3.3).

The reduced-Ls preconditioner replaces z = M^-1 r by z = (T^+ Mhat^-1 T + mu) r,
with M the local operator (+)_s A_s at Ls and Mhat the one at the smaller
extent Ls_hat.  T ((4 Ls_hat) x (4 Ls), spin x fifth dimension, trivial in
colour and space) is trained to minimise

    chi^2(T) = sum_i | M (T^+ Mhat^-1 T + mu) v_i - v_i |^2

over vectors v_i rich in low modes of M (the paper takes the residuals of a
preconditioned solve with the original operators).  With
w = Mhat^-1 T v, e = M (T^+ w + mu v) - v, g = M e and u = Mhat^-1 T g,

    d chi^2 = 2 Re <G, dT>_F,   G = sum_i (w_i g_i^+ + u_i v_i^+),

the outer products contracted over sites and colours.  Along a direction D the
residual is e(eta) = e0 + eta e1 + eta^2 e2 with e1 = M (D^+ w + T^+ y),
e2 = M D^+ y, y = Mhat^-1 D v, so chi^2(T + eta D) is a quartic in eta and the
line search is exact (the real root of its cubic derivative with the lowest
value).  Directions carry momentum (heavy ball, reset to steepest descent when
not a descent direction).  Mhat^-1 is the blocks' inner CG run for a fixed,
large number of iterations (the exact inverse the gradient assumes).

The device backend calls the library for every vector operation (dwf_apply
on the local operator, dwf_reduced_local_inverse, dwf_apply_T,
dwf_T_contract, dwf_field_axpby, dwf_field_dot); torch only holds the device
fields.  What runs on the host is the parameters' own arithmetic: the
(4 Ls_hat) x (4 Ls) matrices T, G and the direction, and the five
coefficients of the line-search quartic.
"""
from __future__ import annotations

import numpy as np


class DeviceBackend:
    """Operators of one lattice handle on canonical FP64 device tensors."""

    def __init__(self, lat, Ls_hat, inverse_iters=60, inner_prec="f32", op_prec="f32"):
        import torch
        from . import binding as B
        from .lattice import PREC
        self.torch, self.B = torch, B
        self.lat, self.Ls, self.Lh = lat, lat.Ls, int(Ls_hat)
        self.iters = int(inverse_iters)
        self.params = B.default_params(inner_prec=PREC[inner_prec])
        self.op_prec = op_prec

    def zeros(self, L):
        return self.torch.zeros((L,) + tuple(self.lat.shape[1:]), dtype=self.torch.complex128, device="cuda")

    def M(self, x):
        B = self.B
        if self.op_prec == "f64":
            return self.lat.apply("local", x.contiguous(), "f64")
        # FP32 operator: the library converts in and out
        xs = self.torch.empty(x.shape, dtype=self.torch.complex64, device="cuda")
        B.dwf_field_axpby(self.lat.h, xs, B.DWF_F32, 1.0, x.contiguous(), in_prec=B.DWF_F64)
        ys = self.lat.apply("local", xs, "f32")
        out = self.zeros(x.shape[0])
        B.dwf_field_axpby(self.lat.h, out, B.DWF_F64, 1.0, ys, in_prec=B.DWF_F32)
        return out

    def Minv_hat(self, x):
        out = self.zeros(self.Lh)
        self.B.dwf_reduced_local_inverse(self.lat.h, out, x.contiguous(), self.Lh, self.iters, self.params)
        return out

    def T(self, T, x, dagger=False):
        out = self.zeros(self.Ls if dagger else self.Lh)
        self.B.dwf_apply_T(self.lat.h, out, x.contiguous(), T, self.Lh, dagger)
        return out

    def contract(self, a, b):
        return self.B.dwf_T_contract(self.lat.h, a.contiguous(), a.shape[0], b.contiguous(), b.shape[0])

    def dot(self, a, b):
        return self.B.dwf_field_dot(self.lat.h, a.contiguous(), b.contiguous(), self.B.DWF_F64, a.shape[0])

    def axpby(self, a, x, b, y):
        """a x + b y (a new field)."""
        out = self.zeros(x.shape[0])
        self.B.dwf_field_axpby(self.lat.h, out, self.B.DWF_F64, a, x.contiguous(), b, y.contiguous(),
                               Ls=x.shape[0])
        return out


class TransformTrainer:
    """chi^2, its gradient and the momentum / exact-line-search descent of
    Sec. 3.3 over a backend (DeviceBackend or any object with the same
    methods)."""

    def __init__(self, backend, vs, mu, momentum=0.5):
        self.be = backend
        self.vs = list(vs)
        self.mu = float(mu)
        self.momentum = float(momentum)
        self.vv = sum(self.be.dot(v, v).real for v in self.vs)

    def _e0(self, T, v):
        be = self.be
        w = be.Minv_hat(be.T(T, v))
        return w, be.axpby(1.0, be.M(be.axpby(1.0, be.T(T, w, dagger=True), self.mu, v)), -1.0, v)

    def loss(self, T):
        """chi^2(T) / sum_i |v_i|^2."""
        return sum(self.be.dot(e, e).real for e in (self._e0(T, v)[1] for v in self.vs)) / self.vv

    def loss_and_grad(self, T):
        """(chi^2 / sum |v|^2, G / sum |v|^2)."""
        be = self.be
        chi2, G = 0.0, np.zeros_like(np.asarray(T, dtype=np.complex128))
        for v in self.vs:
            w, e = self._e0(T, v)
            chi2 += be.dot(e, e).real
            g = be.M(e)
            u = be.Minv_hat(be.T(T, g))
            G = G + be.contract(w, g) + be.contract(u, v)
        return chi2 / self.vv, G / self.vv

    def line_search(self, T, D):
        """eta minimising chi^2(T + eta D) exactly (quartic in eta)."""
        be = self.be
        c = np.zeros(5)
        for v in self.vs:
            w, e0 = self._e0(T, v)
            y = be.Minv_hat(be.T(D, v))
            e1 = be.M(be.axpby(1.0, be.T(D, w, dagger=True), 1.0, be.T(T, y, dagger=True)))
            e2 = be.M(be.T(D, y, dagger=True))
            d00, d11, d22 = be.dot(e0, e0).real, be.dot(e1, e1).real, be.dot(e2, e2).real
            d01, d02, d12 = be.dot(e0, e1).real, be.dot(e0, e2).real, be.dot(e1, e2).real
            c += np.array([d00, 2 * d01, d11 + 2 * d02, 2 * d12, d22])
        # chi^2(eta) = sum_k c[k] eta^k ; stationary points of the quartic
        roots = np.roots([4 * c[4], 3 * c[3], 2 * c[2], c[1]])
        cand = [r.real for r in roots if abs(r.imag) <= 1e-9 * max(1.0, abs(r))]
        quart = lambda eta: sum(c[k] * eta ** k for k in range(5))
        cand = [r for r in cand if r > 0] or [0.0]
        eta = min(cand, key=quart)
        return eta, quart(eta) / self.vv

    def train(self, T0, steps, log=None):
        """Returns (T, history of chi^2 / sum |v|^2 before each step and at the end)."""
        T = np.array(T0, dtype=np.complex128)
        d = np.zeros_like(T)
        hist = []
        for k in range(steps):
            chi2, G = self.loss_and_grad(T)
            hist.append(chi2)
            d = -G + self.momentum * d
            if np.real(np.vdot(G, d)) >= 0:  # not a descent direction: restart
                d = -G
            eta, predicted = self.line_search(T, d)
            T = T + eta * d
            if log:
                log(k, chi2, eta, predicted)
        hist.append(self.loss(T))
        return T, hist
