"""Training the reduced-Ls transform T (Sec. 3.3).

CPU: the trainer's host logic (loss and gradient assembly, the exact quartic
line search, the momentum descent) driven by oracle operators.  GPU: the
device backend's loss and gradient against the oracle's T_loss."""
import numpy as np
import pytest

from paper_2104_05615_gb300 import inputs
from paper_2104_05615_gb300.reduced_ls import TransformTrainer

PAR = dict(b=1.5, c=0.5, M5=1.8)
DIMS, LS, LH, SUB = (8, 2, 2, 2), 4, 2, (4, 2, 2, 2)


class OracleBackend:
    def __init__(self, o, sub, Lh):
        self.o, self.sub, self.Lh = o, sub, Lh

    def M(self, x):
        return self.o.local_DdagD(x, self.sub)

    def Minv_hat(self, x):
        return self.o.reduced_local_inverse(x, self.sub, self.Lh)

    def T(self, T, x, dagger=False):
        return self.o.T_apply(T, x, self.Lh, dagger)

    def contract(self, a, b):
        return self.o.outer_contract(a, b)

    def dot(self, a, b):
        return complex(np.vdot(a, b))

    def axpby(self, a, x, b, y):
        return a * x + b * y


def _setup(orc, seed=3):
    U = inputs.gauge_field(DIMS, 0.5, 11)
    o = orc.Oracle(DIMS, LS, PAR["b"], PAR["c"], PAR["M5"], 0.1, U)
    rng = np.random.default_rng(seed)
    vs = [rng.standard_normal(o.cb_shape()) + 1j * rng.standard_normal(o.cb_shape()) for _ in range(2)]
    T = rng.standard_normal((4 * LH, 4 * LS)) + 1j * rng.standard_normal((4 * LH, 4 * LS))
    return o, vs, 0.3 * T


def test_trainer_loss_and_grad_match_oracle(orc):
    o, vs, T = _setup(orc)
    tr = TransformTrainer(OracleBackend(o, SUB, LH), vs, mu=0.4)
    chi2, G = tr.loss_and_grad(T)
    ref, Gref = o.T_loss(T, 0.4, vs, SUB, LH)
    vv = sum(np.vdot(v, v).real for v in vs)
    assert abs(chi2 - ref / vv) <= 1e-12 * ref / vv
    np.testing.assert_allclose(G, Gref / vv, rtol=0, atol=1e-12 * np.abs(Gref / vv).max())


def test_line_search_quartic_is_exact(orc):
    """chi^2(T + eta D) evaluated directly equals the quartic the line search
    builds, at the chosen eta and at another step."""
    o, vs, T = _setup(orc)
    tr = TransformTrainer(OracleBackend(o, SUB, LH), vs, mu=0.4)
    _, G = tr.loss_and_grad(T)
    eta, pred = tr.line_search(T, -G)
    assert eta > 0
    direct = tr.loss(T - eta * G)
    assert abs(direct - pred) <= 1e-9 * direct
    # a minimum along the line: both neighbours are higher
    assert tr.loss(T - 0.9 * eta * G) >= direct and tr.loss(T - 1.1 * eta * G) >= direct


def test_training_decreases_loss(orc):
    o, vs, T = _setup(orc)
    tr = TransformTrainer(OracleBackend(o, SUB, LH), vs, mu=0.4, momentum=0.5)
    _, hist = tr.train(T, steps=6)
    assert all(b <= a * (1 + 1e-12) for a, b in zip(hist, hist[1:]))
    assert hist[-1] < 0.5 * hist[0]


@pytest.mark.gpu
def test_device_backend_loss_and_gradient_match_oracle(orc):
    torch = pytest.importorskip("torch")
    from paper_2104_05615_gb300.lattice import Lattice, heuristic_T
    from paper_2104_05615_gb300.reduced_ls import DeviceBackend
    dims, Ls, Lh, sub = (8, 4, 4, 4), 8, 4, (4, 4, 4, 4)
    U = inputs.gauge_field(dims, 0.5, 5)
    lat = Lattice(dims, Ls, 1.5, 0.5, 1.8, 0.05, U, sub)
    o = orc.Oracle(dims, Ls, 1.5, 0.5, 1.8, 0.05, U)
    rng = np.random.default_rng(4)
    T = heuristic_T(Ls, Lh) + 0.05 * (rng.standard_normal((4 * Lh, 4 * Ls)) + 1j * rng.standard_normal((4 * Lh, 4 * Ls)))
    vs = [inputs.gaussian_spinor_cb(dims, Ls, 31 + k) for k in range(2)]
    dev = TransformTrainer(DeviceBackend(lat, Lh, inverse_iters=200), [torch.from_numpy(v).cuda() for v in vs], mu=0.3)
    chi2, G = dev.loss_and_grad(T)
    ref, Gref = o.T_loss(T, 0.3, vs, sub, Lh)
    vv = sum(np.vdot(v, v).real for v in vs)
    assert abs(chi2 - ref / vv) <= 1e-4 * ref / vv
    assert np.linalg.norm(G - Gref / vv) <= 1e-3 * np.linalg.norm(Gref / vv)
