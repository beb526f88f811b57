"""ctypes binding of the C ABI in include/dwf.h (argument marshalling only).

Every function keeps the C name and forwards to libdwf_gb300.so; tensors are
passed as raw device (or host) pointers.  There is no fallback: if the library
is missing the import of a function raises.
"""
from __future__ import annotations

import ctypes as C
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libdwf_gb300.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "dwf.h")

DWF_OK, DWF_EINVAL, DWF_ENOMEM, DWF_ECUDA, DWF_ENOCONV, DWF_ETIMEOUT, DWF_EUNSUPPORTED = range(7)
DWF_F64, DWF_F32, DWF_F16, DWF_BF16, DWF_FX16, DWF_FX8 = range(6)
DWF_OP_D, DWF_OP_DDAG, DWF_OP_DDAGD, DWF_OP_LOCAL_DDAGD, DWF_OP_M5INV, DWF_OP_M5INVDAG = range(6)


class dwf_solver_params(C.Structure):
    _fields_ = [("tol", C.c_double), ("maxiter", C.c_int), ("inner_iters", C.c_int),
                ("outer_prec", C.c_int), ("inner_prec", C.c_int), ("delta", C.c_double),
                ("use_reduced_ls", C.c_int), ("use_graph", C.c_int), ("check_every", C.c_int),
                ("time_kernels", C.c_int), ("precond_wave", C.c_int)]


class dwf_geometry(C.Structure):
    _fields_ = [(n, C.c_longlong) for n in (
        "even_sites", "even_sites_padded", "blocks", "block_sites", "block_sites_padded",
        "o1_sites", "o1_sites_padded", "e2_sites", "e2_sites_padded")]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class dwf_kernel_config(C.Structure):
    _fields_ = [("tile_sites", C.c_int), ("gather", C.c_int)]


class dwf_stats(C.Structure):
    _fields_ = [("outer_iters", C.c_int), ("inner_iters_total", C.c_int),
                ("reliable_updates", C.c_int), ("converged", C.c_int),
                ("true_residual", C.c_double), ("time_total_ms", C.c_double),
                ("kernel_launches", C.c_longlong), ("local_op_ms", C.c_double),
                ("local_op_count", C.c_longlong), ("outer_op_ms", C.c_double),
                ("outer_op_count", C.c_longlong)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def lib() -> C.CDLL:
    """Load the CUDA library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built: {LIB_PATH} (run __graft_entry__.build())")
        L = C.CDLL(LIB_PATH)
        vp, i, d = C.c_void_p, C.c_int, C.c_double
        sig = {
            "dwf_default_params": (None, [C.POINTER(dwf_solver_params)]),
            "dwf_create": (i, [C.POINTER(vp), vp, C.POINTER(C.c_int), i, d, d, d, d,
                               C.POINTER(C.c_int), i, vp]),
            "dwf_destroy": (None, [vp]),
            "dwf_last_error": (C.c_char_p, [vp]),
            "dwf_status_string": (C.c_char_p, [i]),
            "dwf_field_elems": (C.c_size_t, [vp, i]),
            "dwf_packed_bytes": (C.c_size_t, [vp, i, i]),
            "dwf_pack": (i, [vp, vp, vp, i, vp]),
            "dwf_unpack": (i, [vp, vp, vp, i, vp]),
            "dwf_apply": (i, [vp, vp, vp, i, i, vp]),
            "dwf_apply_packed": (i, [vp, vp, vp, i, i, vp]),
            "dwf_cg": (i, [vp, vp, vp, C.POINTER(dwf_solver_params), C.POINTER(dwf_stats)]),
            "dwf_mspcg": (i, [vp, vp, vp, C.POINTER(dwf_solver_params), C.POINTER(dwf_stats)]),
            "dwf_solve_host": (i, [vp, vp, vp, C.POINTER(dwf_solver_params), i,
                                   C.POINTER(dwf_stats)]),
            "dwf_precondition": (i, [vp, vp, vp, C.POINTER(dwf_solver_params)]),
            "dwf_set_reduced_ls": (i, [vp, i, vp, d]),
            "dwf_set_local_truncated": (i, [vp, i]),
            "dwf_reduced_local_inverse": (i, [vp, vp, vp, i, i, C.POINTER(dwf_solver_params)]),
            "dwf_apply_T": (i, [vp, vp, vp, vp, i, i]),
            "dwf_T_contract": (i, [vp, vp, vp, i, vp, i]),
            "dwf_batch_create": (i, [C.POINTER(vp), C.POINTER(vp), i]),
            "dwf_batch_destroy": (None, [vp]),
            "dwf_batch_mspcg": (i, [vp, C.POINTER(vp), C.POINTER(vp),
                                    C.POINTER(dwf_solver_params), C.POINTER(dwf_stats),
                                    C.POINTER(dwf_stats)]),
            "dwf_batch_last_error": (C.c_char_p, [vp]),
            "dwf_kernel_launch_count": (C.c_longlong, []),
            "dwf_get_geometry": (i, [vp, C.POINTER(dwf_geometry)]),
            "dwf_autotune": (i, [vp, i, i]),
            "dwf_apply_packed_static": (i, [vp, vp, vp, i, i, vp]),
            "dwf_get_kernel_config": (i, [vp, i, i, C.POINTER(dwf_kernel_config)]),
            "dwf_set_kernel_config": (i, [vp, i, i, C.POINTER(dwf_kernel_config)]),
            "dwf_fma_peak": (i, [vp, i, C.POINTER(C.c_double)]),
            "dwf_query_geometry": (i, [C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(dwf_geometry)]),
            "dwf_set_wait_policy": (i, [vp, C.c_longlong, i]),
            "dwf_field_axpby": (i, [vp, vp, i, d, d, vp, d, d, vp, i, i]),
            "dwf_field_dot": (i, [vp, C.POINTER(C.c_double), vp, vp, i, i]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def header_functions():
    """Function names declared in include/dwf.h."""
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(dwf_[a-z0-9_]+)\s*\(", txt)))


class DwfError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{lib().dwf_status_string(status).decode()} ({status}): {msg}")
        self.status = status


def check(status, handle=None, batch=None):
    if status != DWF_OK:
        msg = ""
        if handle is not None:
            msg = lib().dwf_last_error(handle).decode()
        elif batch is not None:
            msg = lib().dwf_batch_last_error(batch).decode()
        raise DwfError(status, msg)
    return status


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if hasattr(t, "data_ptr"):
        return t.data_ptr()
    if hasattr(t, "ctypes"):
        return t.ctypes.data
    raise TypeError(type(t))


def _stream(s):
    if s is None:
        return None
    if hasattr(s, "cuda_stream"):
        return s.cuda_stream
    return int(s)


def default_params(**kw) -> dwf_solver_params:
    p = dwf_solver_params()
    lib().dwf_default_params(C.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def dwf_create(gauge_host, dims, Ls, b, c, M5, mass, subdomain=None, t_antiperiodic=0,
               stream=None):
    h = C.c_void_p()
    dims_a = (C.c_int * 4)(*dims)
    sub_a = None if subdomain is None else (C.c_int * 4)(*subdomain)
    st = lib().dwf_create(C.byref(h), _ptr(gauge_host), dims_a, int(Ls), float(b), float(c),
                          float(M5), float(mass), sub_a, int(t_antiperiodic), _stream(stream))
    check(st)
    return h


def dwf_destroy(h):
    lib().dwf_destroy(h)


def dwf_apply(h, out, inp, op, prec, stream=None):
    return check(lib().dwf_apply(h, _ptr(out), _ptr(inp), int(op), int(prec), _stream(stream)), h)


def dwf_apply_packed(h, out, inp, op, prec, stream=None):
    return check(lib().dwf_apply_packed(h, _ptr(out), _ptr(inp), int(op), int(prec),
                                        _stream(stream)), h)


def dwf_apply_packed_static(h, out, inp, op, prec, stream=None):
    return check(lib().dwf_apply_packed_static(h, _ptr(out), _ptr(inp), int(op), int(prec),
                                               _stream(stream)), h)


def dwf_pack(h, packed, canon, prec, stream=None):
    return check(lib().dwf_pack(h, _ptr(packed), _ptr(canon), int(prec), _stream(stream)), h)


def dwf_unpack(h, canon, packed, prec, stream=None):
    return check(lib().dwf_unpack(h, _ptr(canon), _ptr(packed), int(prec), _stream(stream)), h)


def dwf_packed_bytes(h, prec, Ls=0):
    return lib().dwf_packed_bytes(h, int(prec), int(Ls))


def dwf_field_elems(h, Ls=0):
    return lib().dwf_field_elems(h, int(Ls))


def _solve(fn, h, x, b, params, raise_on_noconv):
    st = dwf_stats()
    p = params if params is not None else default_params()
    s = fn(h, _ptr(x), _ptr(b), C.byref(p), C.byref(st))
    if s != DWF_ENOCONV or raise_on_noconv:
        check(s, h)
    return st, s


def dwf_cg(h, x, b, params=None, raise_on_noconv=True):
    return _solve(lib().dwf_cg, h, x, b, params, raise_on_noconv)[0]


def dwf_mspcg(h, x, b, params=None, raise_on_noconv=True):
    return _solve(lib().dwf_mspcg, h, x, b, params, raise_on_noconv)[0]


def dwf_solve_host(h, x_host, b_host, params=None, use_mspcg=True):
    st = dwf_stats()
    p = params if params is not None else default_params()
    check(lib().dwf_solve_host(h, _ptr(x_host), _ptr(b_host), C.byref(p), int(use_mspcg),
                               C.byref(st)), h)
    return st


def dwf_precondition(h, z, r, params=None):
    p = params if params is not None else default_params()
    return check(lib().dwf_precondition(h, _ptr(z), _ptr(r), C.byref(p)), h)


def dwf_set_reduced_ls(h, Ls_hat, T_host, mu):
    return check(lib().dwf_set_reduced_ls(h, int(Ls_hat), _ptr(T_host), float(mu)), h)


def dwf_set_local_truncated(h, on):
    return check(lib().dwf_set_local_truncated(h, int(bool(on))), h)


def dwf_reduced_local_inverse(h, out, inp, Ls_hat, iters, params=None):
    """out = CG_iters(Mhat) inp on canonical FP64 device tensors (Ls_hat slices)."""
    p = params if params is not None else default_params()
    return check(lib().dwf_reduced_local_inverse(h, _ptr(out), _ptr(inp), int(Ls_hat), int(iters),
                                                 C.byref(p)), h)


def dwf_apply_T(h, out, inp, T_host, Ls_hat, dagger=False):
    """out = T inp (dagger False) or T^+ inp on canonical FP64 device tensors."""
    import numpy as np
    T = np.ascontiguousarray(T_host, dtype=np.complex128)
    return check(lib().dwf_apply_T(h, _ptr(out), _ptr(inp), _ptr(T), int(Ls_hat), int(bool(dagger))), h)


def dwf_T_contract(h, a, La, b, Lb):
    """sum over sites and colours of a b^+ as a (4 La) x (4 Lb) complex numpy matrix."""
    import numpy as np
    G = np.empty((4 * La, 4 * Lb), dtype=np.complex128)
    check(lib().dwf_T_contract(h, _ptr(G), _ptr(a), int(La), _ptr(b), int(Lb)), h)
    return G


def dwf_batch_create(handles):
    bt = C.c_void_p()
    arr = (C.c_void_p * len(handles))(*[h.value for h in handles])
    check(lib().dwf_batch_create(C.byref(bt), arr, len(handles)))
    return bt


def dwf_batch_destroy(bt):
    lib().dwf_batch_destroy(bt)


def dwf_batch_mspcg(bt, xs, bs, params=None):
    n = len(xs)
    xa = (C.c_void_p * n)(*[_ptr(x) for x in xs])
    ba = (C.c_void_p * n)(*[_ptr(b) for b in bs])
    per = (dwf_stats * n)()
    tot = dwf_stats()
    p = params if params is not None else default_params()
    check(lib().dwf_batch_mspcg(bt, xa, ba, C.byref(p), per, C.byref(tot)), batch=bt)
    return tot, list(per)


def dwf_get_geometry(h):
    g = dwf_geometry()
    check(lib().dwf_get_geometry(h, C.byref(g)), h)
    return g.as_dict()


def dwf_query_geometry(dims, sub=None):
    """Site counts of a lattice and block dims without a handle or a device."""
    g = dwf_geometry()
    d = (C.c_int * 4)(*[int(v) for v in dims])
    sb = (C.c_int * 4)(*[int(v) for v in sub]) if sub is not None else None
    check(lib().dwf_query_geometry(d, sb, C.byref(g)))
    return g.as_dict()


def dwf_autotune(h, prec, op_kind):
    return check(lib().dwf_autotune(h, int(prec), int(op_kind)), h)


def dwf_get_kernel_config(h, prec, op_kind):
    c = dwf_kernel_config()
    check(lib().dwf_get_kernel_config(h, int(prec), int(op_kind), C.byref(c)), h)
    return {"tile_sites": c.tile_sites, "gather": c.gather}


def dwf_set_kernel_config(h, prec, op_kind, tile_sites, gather):
    c = dwf_kernel_config(int(tile_sites), int(gather))
    return check(lib().dwf_set_kernel_config(h, int(prec), int(op_kind), C.byref(c)), h)


def dwf_set_wait_policy(h, max_polls=0, force_timeout=False):
    """Poll limit of the bounded device waits (0: default) and the test-only
    forced time-out of the bulk-copy stage kernels."""
    return check(lib().dwf_set_wait_policy(h, int(max_polls), int(bool(force_timeout))), h)


def dwf_field_axpby(h, out, out_prec, a, x, b=0.0, y=None, in_prec=None, Ls=0):
    """out = a x + b y on canonical device fields (complex a, b; y None: a x)."""
    a, b = complex(a), complex(b)
    in_prec = out_prec if in_prec is None else in_prec
    return check(lib().dwf_field_axpby(h, _ptr(out), int(out_prec), a.real, a.imag, _ptr(x), b.real, b.imag,
                                       _ptr(y), int(in_prec), int(Ls)), h)


def dwf_field_dot(h, a, b, prec, Ls=0):
    """<a, b> = sum conj(a) b of canonical device fields, FP64, fixed-order sums."""
    r = (C.c_double * 2)()
    check(lib().dwf_field_dot(h, r, _ptr(a), _ptr(b), int(prec), int(Ls)), h)
    return complex(r[0], r[1])


def dwf_kernel_launch_count():
    return lib().dwf_kernel_launch_count()


def dwf_fma_peak(h, prec):
    """Measured CUDA-core FMA rate (TFLOP/s) in DWF_F32 or DWF_F64."""
    v = C.c_double()
    check(lib().dwf_fma_peak(h, int(prec), C.byref(v)), h)
    return v.value
