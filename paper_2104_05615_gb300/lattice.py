"""Convenience wrapper over the C ABI for one lattice, with torch device tensors.

Canonical even/odd fields are torch tensors of shape (Ls, V/2, 4, 3):
complex128 (FP64), complex64 (FP32 and the 16- and 8-bit fixed-point formats,
device storage formats exchanged as FP32); FP16 / BF16 fields carry a
trailing (re, im) axis: float16 / bfloat16 of shape (Ls, V/2, 4, 3, 2).
"""
from __future__ import annotations

import numpy as np
import torch

from . import binding as B
from . import inputs

PREC = {"f64": B.DWF_F64, "f32": B.DWF_F32, "f16": B.DWF_F16, "bf16": B.DWF_BF16,
        "fx16": B.DWF_FX16, "fx8": B.DWF_FX8}
OPS = {"D": B.DWF_OP_D, "Ddag": B.DWF_OP_DDAG, "DdagD": B.DWF_OP_DDAGD,
       "local": B.DWF_OP_LOCAL_DDAGD, "m5inv": B.DWF_OP_M5INV, "m5invdag": B.DWF_OP_M5INVDAG}


def to_device(x: np.ndarray, prec: str, device="cuda") -> torch.Tensor:
    """numpy complex128 (Ls, Vh, 4, 3) -> canonical torch tensor of a precision."""
    t = torch.from_numpy(np.ascontiguousarray(x))
    if prec == "f64":
        return t.to(device)
    if prec in ("f32", "fx16", "fx8"):
        return t.to(torch.complex64).to(device)
    r = torch.view_as_real(t.to(torch.complex64))
    return r.to(torch.float16 if prec == "f16" else torch.bfloat16).to(device).contiguous()


def to_numpy(t: torch.Tensor) -> np.ndarray:
    if t.dtype in (torch.float16, torch.bfloat16):
        t = torch.view_as_complex(t.float().contiguous())
    return t.detach().cpu().to(torch.complex128).numpy()


def empty_like_prec(shape, prec, device="cuda"):
    if prec == "f64":
        return torch.empty(shape, dtype=torch.complex128, device=device)
    if prec in ("f32", "fx16", "fx8"):
        return torch.empty(shape, dtype=torch.complex64, device=device)
    return torch.empty(tuple(shape) + (2,), dtype=torch.float16 if prec == "f16" else torch.bfloat16,
                       device=device)


class Lattice:
    """One lattice and its handle."""

    def __init__(self, dims, Ls, b, c, M5, mass, gauge, sub=None, antiperiodic_t=0, stream=None):
        self.dims = tuple(int(d) for d in dims)
        self.Ls = int(Ls)
        self.V = int(np.prod(self.dims))
        self.Vh = self.V // 2
        self.gauge = np.ascontiguousarray(gauge, dtype=np.complex128)
        self.sub = tuple(sub) if sub is not None else self.dims
        self.h = B.dwf_create(self.gauge, self.dims, self.Ls, b, c, M5, mass, self.sub,
                              antiperiodic_t, stream)
        self.params = dict(b=b, c=c, M5=M5, mass=mass)

    @classmethod
    def from_config(cls, cfg, stream=None):
        U = inputs.gauge_field(cfg["dims"], cfg["eps"], cfg["gauge_seed"])
        return cls(cfg["dims"], cfg["Ls"], cfg["b"], cfg["c"], cfg["M5"], cfg["mass"], U,
                   cfg.get("sub"), 0, stream)

    def close(self):
        if self.h is not None:
            B.dwf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def shape(self):
        return (self.Ls, self.Vh, 4, 3)

    def apply(self, op: str, x: torch.Tensor, prec: str = "f64", out=None, stream=None):
        out = empty_like_prec(self.shape, prec) if out is None else out
        B.dwf_apply(self.h, out, x, OPS[op], PREC[prec], stream)
        return out

    def packed(self, prec: str, Ls: int = 0) -> torch.Tensor:
        n = B.dwf_packed_bytes(self.h, PREC[prec], Ls)
        return torch.zeros(n, dtype=torch.uint8, device="cuda")

    def pack(self, x, prec, stream=None):
        p = self.packed(prec)
        B.dwf_pack(self.h, p, x, PREC[prec], stream)
        return p

    def unpack(self, p, prec, stream=None):
        out = empty_like_prec(self.shape, prec)
        B.dwf_unpack(self.h, out, p, PREC[prec], stream)
        return out

    def solve(self, b: torch.Tensor, x0=None, mspcg=True, raise_on_noconv=True, **params):
        x = torch.zeros_like(b) if x0 is None else x0.clone()
        p = B.default_params(**{k: (PREC[v] if k.endswith("_prec") and isinstance(v, str) else v)
                                for k, v in params.items()})
        fn = B.dwf_mspcg if mspcg else B.dwf_cg
        st = fn(self.h, x, b, p, raise_on_noconv=raise_on_noconv)
        return x, st.as_dict()

    def set_reduced_ls(self, Ls_hat, T: np.ndarray, mu: float):
        T = np.ascontiguousarray(T, dtype=np.complex128)
        B.dwf_set_reduced_ls(self.h, Ls_hat, T, mu)
        self._T = T


def heuristic_T(Ls: int, Ls_hat: int) -> np.ndarray:
    """Fifth-dimension map that keeps the Ls_hat/2 slices next to each wall
    (spin identity): slices 0..h-1 -> 0..h-1 and Ls-h..Ls-1 -> Ls_hat-h..Ls_hat-1."""
    h = Ls_hat // 2
    T = np.zeros((4 * Ls_hat, 4 * Ls), dtype=np.complex128)
    for s in range(h):
        for a in range(4):
            T[s * 4 + a, s * 4 + a] = 1.0
            T[(Ls_hat - 1 - s) * 4 + a, (Ls - 1 - s) * 4 + a] = 1.0
    return T
