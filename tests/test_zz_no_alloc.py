"""The allocation-free operator entry point, dwf_apply_packed_static.

Some callers cannot allocate device memory when they apply the operator: code
whose device memory is all owned by an arena or pool, callers that must not
touch the allocator while other work is in flight, and hosts that forbid
allocation after start-up.  dwf_apply_packed_static serves them by keeping its
three intermediate fields in a fixed file-scope device array.  These tests
check, through the C ABI, that it gives the same D^+D (and D, D^+) as the
ordinary dwf_apply_packed on two calls in a row in every storage format, that
the calls take no device memory (the device's free memory is unchanged across
them), and that a lattice just inside the array's size is served while one
just beyond it is refused.  This file is collected last on purpose.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2104_05615_gb300 import inputs  # noqa: E402

# the accuracy each storage format allows (as in the operator parity tests);
# both entry points run the same kernels, so they agree far inside these
TOL = {"f64": 1e-12, "f32": 1e-6, "f16": 5e-3, "bf16": 5e-3, "fx16": 5e-3, "fx8": 3e-2}
SCRATCH_BYTES = 24 << 20


def _lattice(dims=(8, 4, 4, 4), Ls=8, sub=(4, 4, 4, 4)):
    from paper_2104_05615_gb300.lattice import Lattice
    U = inputs.gauge_field(dims, 0.5, 23)
    return Lattice(dims, Ls, 1.5, 0.5, 1.8, 0.03, U, sub)


def _check_same_as_allocating(lat, prec):
    from paper_2104_05615_gb300 import binding as B
    from paper_2104_05615_gb300.lattice import PREC, to_device, to_numpy
    x = to_device(inputs.gaussian_spinor_cb(lat.dims, lat.Ls, 31), prec)
    xin = lat.pack(x, prec)
    for op in (B.DWF_OP_DDAGD, B.DWF_OP_D, B.DWF_OP_DDAG):
        ref = lat.packed(prec)
        # the ordinary entry point (it also builds what the static one needs)
        B.dwf_apply_packed(lat.h, ref, xin, op, PREC[prec])
        want = to_numpy(lat.unpack(ref, prec))
        outs = [lat.packed(prec) for _ in range(3)]
        # the first call on a device may load the module that holds the array
        B.dwf_apply_packed_static(lat.h, outs[0], xin, op, PREC[prec])
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        for out in outs[1:]:  # two calls in a row share the static array
            B.dwf_apply_packed_static(lat.h, out, xin, op, PREC[prec])
        torch.cuda.synchronize()
        # the calls allocated nothing on the device
        assert torch.cuda.mem_get_info()[0] == free0, op
        for out in outs:
            got = to_numpy(lat.unpack(out, prec))
            err = np.linalg.norm(got - want) / np.linalg.norm(want)
            assert err <= TOL[prec], (op, err)


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["f64", "f32", "f16", "bf16", "fx16", "fx8"])
def test_static_scratch_matches_allocating_entry_point(prec):
    _check_same_as_allocating(_lattice(), prec)


@pytest.mark.gpu
def test_static_scratch_size_limit():
    from paper_2104_05615_gb300 import binding as B
    lat = _lattice(dims=(12, 12, 12, 12), Ls=12, sub=None)
    # FP16 on 12^4 x Ls = 12: three fields of 6.5 MB fit in the 24 MiB array
    assert 3 * B.dwf_packed_bytes(lat.h, B.DWF_F16, 0) <= SCRATCH_BYTES
    _check_same_as_allocating(lat, "f16")
    # FP32 on the same lattice: three fields of 11.9 MB do not
    assert 3 * B.dwf_packed_bytes(lat.h, B.DWF_F32, 0) > SCRATCH_BYTES
    B.dwf_apply_packed(lat.h, lat.packed("f32"), lat.packed("f32"), B.DWF_OP_DDAGD, B.DWF_F32)
    x = lat.packed("f32")
    out = lat.packed("f32")
    with pytest.raises(B.DwfError) as e:
        B.dwf_apply_packed_static(lat.h, out, x, B.DWF_OP_DDAGD, B.DWF_F32)
    assert e.value.status == B.DWF_EINVAL
