"""Failure detection on the GPU without a fault: the bounded device waits of the
bulk-copy stage kernels give up, raise the handle's error flag, and the call
reports DWF_ETIMEOUT; the handle then works normally again.

The wait is made to run out by dwf_set_wait_policy's test setting: every copy
of the kernel lands as usual, then each CTA waits on an mbarrier phase that is
never armed, with a short poll limit.  Nothing is in flight when it gives up,
nothing traps, and nothing hangs.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2104_05615_gb300 import inputs  # noqa: E402


def relerr(a, b):
    return np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel())


@pytest.mark.gpu
@pytest.mark.parametrize("op,kind", [("local", 1), ("DdagD", 0)])
def test_bounded_wait_times_out_and_handle_recovers(orc, op, kind):
    from paper_2104_05615_gb300 import binding as B
    from paper_2104_05615_gb300.lattice import Lattice, to_device, to_numpy
    dims, Ls, sub = (8, 4, 4, 4), 8, (4, 4, 4, 4)
    U = inputs.gauge_field(dims, 0.5, 41)
    lat = Lattice(dims, Ls, 1.5, 0.5, 1.8, 0.03, U, sub)
    o = orc.Oracle(dims, Ls, 1.5, 0.5, 1.8, 0.03, U)
    x = inputs.gaussian_spinor_cb(dims, Ls, 42)
    xd = to_device(x, "f32")
    want = o.local_DdagD(to_numpy(xd), sub) if op == "local" else o.DdagD(to_numpy(xd))
    # the bulk-copy gather (the kernels with an mbarrier wait)
    B.dwf_set_kernel_config(lat.h, B.DWF_F32, kind, 8, 1)
    B.dwf_set_wait_policy(lat.h, 1 << 12, True)
    with pytest.raises(B.DwfError) as e:
        lat.apply(op, xd, "f32")
    assert e.value.status == B.DWF_ETIMEOUT
    # back to normal: the same call succeeds and is correct, twice
    B.dwf_set_wait_policy(lat.h, 0, False)
    for _ in range(2):
        got = to_numpy(lat.apply(op, xd, "f32"))
        assert relerr(got, want) < 1e-6
    torch.cuda.synchronize()
