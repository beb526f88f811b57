"""The vector calls on canonical fields (dwf_field_axpby, dwf_field_dot) that
the transform training of Sec. 3.3 assembles its loss from: element-wise
results against numpy, the FP64 inner product against numpy's, the same bits
on every call, and the FP64 -> FP32 cast equal to numpy's rounding."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2104_05615_gb300 import inputs  # noqa: E402


@pytest.mark.gpu
def test_field_axpby_and_dot():
    from paper_2104_05615_gb300 import binding as B
    from paper_2104_05615_gb300.lattice import Lattice
    dims, Ls = (8, 4, 4, 4), 8
    lat = Lattice(dims, Ls, 1.5, 0.5, 1.8, 0.05, inputs.gauge_field(dims, 0.5, 3), (4, 4, 4, 4))
    x = inputs.gaussian_spinor_cb(dims, Ls, 61)
    y = inputs.gaussian_spinor_cb(dims, Ls, 62)
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    a, b = 0.7 - 0.2j, -1.3 + 0.4j
    out = torch.empty_like(xd)
    B.dwf_field_axpby(lat.h, out, B.DWF_F64, a, xd, b, yd)
    np.testing.assert_allclose(out.cpu().numpy(), a * x + b * y, rtol=0, atol=1e-14 * np.abs(x).max() * 4)
    # in place (out = y) and y = None
    B.dwf_field_axpby(lat.h, yd, B.DWF_F64, 1.0, xd, 2.0, yd)
    np.testing.assert_allclose(yd.cpu().numpy(), x + 2.0 * y, rtol=0, atol=1e-13)
    B.dwf_field_axpby(lat.h, out, B.DWF_F64, 3.0, xd)
    np.testing.assert_allclose(out.cpu().numpy(), 3.0 * x, rtol=0, atol=1e-13)
    # the cast rounds like numpy
    xs = torch.empty(xd.shape, dtype=torch.complex64, device="cuda")
    B.dwf_field_axpby(lat.h, xs, B.DWF_F32, 1.0, xd, in_prec=B.DWF_F64)
    assert np.array_equal(xs.cpu().numpy(), x.astype(np.complex64))
    # FP64 inner product, fixed-order sums
    yd = torch.from_numpy(y).cuda()
    d1 = B.dwf_field_dot(lat.h, xd, yd, B.DWF_F64)
    d2 = B.dwf_field_dot(lat.h, xd, yd, B.DWF_F64)
    ref = np.vdot(x, y)
    assert abs(d1 - ref) <= 1e-12 * abs(ref) and d1 == d2
    ds = B.dwf_field_dot(lat.h, xs, xs, B.DWF_F32)
    xs64 = x.astype(np.complex64).astype(np.complex128)
    assert abs(ds - np.vdot(xs64, xs64)) <= 1e-12 * np.vdot(xs64, xs64).real
