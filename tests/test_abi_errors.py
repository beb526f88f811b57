"""Error behaviour of the C ABI that needs no GPU: every entry point given a
null handle (or batch) returns DWF_EINVAL, and dwf_create rejects bad lattice
arguments while validating them on the host, before any device work."""
import ctypes as C

import numpy as np
import pytest

from paper_2104_05615_gb300 import binding as B


@pytest.fixture(scope="module")
def lib():
    return B.lib()


def test_status_strings_and_defaults(lib):
    for s in range(0, 7):
        assert lib.dwf_status_string(s)
    p = B.dwf_solver_params()
    lib.dwf_default_params(C.byref(p))
    assert 0 < p.tol < 1 and p.inner_iters >= 1 and p.maxiter > 0
    assert lib.dwf_kernel_launch_count() >= 0


def test_null_handle_is_rejected(lib):
    E = B.DWF_EINVAL
    p = B.default_params()
    st = B.dwf_stats()
    kc = B.dwf_kernel_config(8, 0)
    g = B.dwf_geometry()
    calls = {
        "dwf_get_geometry": (None, C.byref(g)),
        "dwf_pack": (None, None, None, B.DWF_F32, None),
        "dwf_unpack": (None, None, None, B.DWF_F32, None),
        "dwf_apply": (None, None, None, B.DWF_OP_DDAGD, B.DWF_F32, None),
        "dwf_apply_packed": (None, None, None, B.DWF_OP_DDAGD, B.DWF_F32, None),
        "dwf_apply_packed_static": (None, None, None, B.DWF_OP_DDAGD, B.DWF_F32, None),
        "dwf_cg": (None, None, None, C.byref(p), C.byref(st)),
        "dwf_mspcg": (None, None, None, C.byref(p), C.byref(st)),
        "dwf_solve_host": (None, None, None, C.byref(p), 1, C.byref(st)),
        "dwf_precondition": (None, None, None, C.byref(p)),
        "dwf_set_reduced_ls": (None, 4, None, 0.5),
        "dwf_set_local_truncated": (None, 1),
        "dwf_reduced_local_inverse": (None, None, None, 4, 10, C.byref(p)),
        "dwf_apply_T": (None, None, None, None, 4, 0),
        "dwf_T_contract": (None, None, None, 4, None, 8),
        "dwf_autotune": (None, B.DWF_F32, 0),
        "dwf_get_kernel_config": (None, B.DWF_F32, 0, C.byref(kc)),
        "dwf_set_kernel_config": (None, B.DWF_F32, 0, C.byref(kc)),
        "dwf_batch_mspcg": (None, None, None, C.byref(p), None, C.byref(st)),
        "dwf_set_wait_policy": (None, 0, 0),
        "dwf_field_axpby": (None, None, B.DWF_F64, 1.0, 0.0, None, 0.0, 0.0, None, B.DWF_F64, 0),
        "dwf_field_dot": (None, None, None, None, B.DWF_F64, 0),
    }
    for name, args in calls.items():
        assert getattr(lib, name)(*args) == E, name
    assert lib.dwf_field_elems(None, 0) == 0
    assert lib.dwf_packed_bytes(None, B.DWF_F32, 0) == 0
    assert lib.dwf_last_error(None) and lib.dwf_batch_last_error(None)
    lib.dwf_destroy(None)
    lib.dwf_batch_destroy(None)


def _create(lib, dims, Ls=8, sub=None):
    h = C.c_void_p()
    V = int(np.prod(dims))
    U = np.zeros((V, 4, 3, 3, 2))
    d = (C.c_int * 4)(*dims)
    s = (C.c_int * 4)(*(sub or dims))
    return lib.dwf_create(C.byref(h), U.ctypes.data, d, Ls, 1.5, 0.5, 1.8, 0.01, s, 0, None), h


def test_create_rejects_bad_lattices_on_the_host(lib):
    E = B.DWF_EINVAL
    h = C.c_void_p()
    d = (C.c_int * 4)(4, 4, 4, 4)
    U = np.zeros(256 * 4 * 18)
    assert lib.dwf_create(None, U.ctypes.data, d, 8, 1.5, 0.5, 1.8, 0.01, None, 0, None) == E
    assert lib.dwf_create(C.byref(h), None, d, 8, 1.5, 0.5, 1.8, 0.01, None, 0, None) == E
    assert _create(lib, (4, 4, 4, 4), Ls=0)[0] == E                       # Ls out of range
    assert _create(lib, (4, 4, 4, 4), Ls=33)[0] == E
    assert _create(lib, (5, 4, 4, 4))[0] == E                             # odd extent
    assert _create(lib, (8, 4, 4, 4), sub=(3, 4, 4, 4))[0] == E           # block does not divide
    assert _create(lib, (8, 4, 4, 4), sub=(6, 4, 4, 4))[0] == E
    assert _create(lib, (6, 4, 4, 4), sub=(4, 4, 4, 4))[0] == E
    assert _create(lib, (4, 4, 4, 4), sub=(2, 4, 4, 4))[0] == E           # lattice - block < 4
    bt = C.c_void_p()
    assert lib.dwf_batch_create(C.byref(bt), None, 2) == E
    assert lib.dwf_batch_create(None, None, 0) == E
