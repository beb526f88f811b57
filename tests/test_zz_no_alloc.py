"""The allocation-free operator entry point, dwf_apply_packed_static.

Some callers cannot allocate device memory when they apply the operator: code
whose device memory is all owned by an arena or pool, callers that must not
touch the allocator while other work is in flight, and hosts that forbid
allocation after start-up.  dwf_apply_packed_static serves them by keeping its
three intermediate fields in a fixed file-scope device array.  These tests
check, through the C ABI, that it gives the same D^+D (and D, D^+) as the
ordinary dwf_apply_packed on two calls in a row, and that lattices too large
for the array are refused.  This file is collected last on purpose.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2104_05615_gb300 import inputs  # noqa: E402

TOL = {"f32": 1e-6, "f16": 5e-3}


def _lattice(dims=(8, 4, 4, 4), Ls=8, sub=(4, 4, 4, 4)):
    from paper_2104_05615_gb300.lattice import Lattice
    U = inputs.gauge_field(dims, 0.5, 23)
    return Lattice(dims, Ls, 1.5, 0.5, 1.8, 0.03, U, sub)


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["f32", "f16"])
def test_static_scratch_matches_allocating_entry_point(prec):
    from paper_2104_05615_gb300 import binding as B
    from paper_2104_05615_gb300.lattice import PREC, to_device, to_numpy
    lat = _lattice()
    x = to_device(inputs.gaussian_spinor_cb(lat.dims, lat.Ls, 31), prec)
    xin = lat.pack(x, prec)
    for op in (B.DWF_OP_DDAGD, B.DWF_OP_D, B.DWF_OP_DDAG):
        ref = lat.packed(prec)
        # the ordinary entry point (it also builds what the static one needs)
        B.dwf_apply_packed(lat.h, ref, xin, op, PREC[prec])
        want = to_numpy(lat.unpack(ref, prec))
        for _ in range(2):  # two calls in a row share the static array
            out = lat.packed(prec)
            B.dwf_apply_packed_static(lat.h, out, xin, op, PREC[prec])
            got = to_numpy(lat.unpack(out, prec))
            err = np.linalg.norm(got - want) / np.linalg.norm(want)
            assert err <= TOL[prec], (op, err)
    torch.cuda.synchronize()


@pytest.mark.gpu
def test_static_scratch_refuses_too_large_lattice():
    from paper_2104_05615_gb300 import binding as B
    # 16^4 x Ls=16 in FP32: three intermediate fields of 50 MB each > 24 MiB
    lat = _lattice(dims=(16, 16, 16, 16), Ls=16, sub=(8, 8, 8, 8))
    x = lat.packed("f32")
    out = lat.packed("f32")
    with pytest.raises(B.DwfError) as e:
        B.dwf_apply_packed_static(lat.h, out, x, B.DWF_OP_DDAGD, B.DWF_F32)
    assert e.value.status == B.DWF_EINVAL
