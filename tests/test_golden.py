"""Stored expected values (tests/golden/, written by tests/golden/make_golden.py
from the oracle alone): M5op^-1 of Sec. 2.2 at the 16^3x32 workload's
fifth-dimension parameters.  The oracle must keep reproducing them (CPU), and
the library's FP64 M5^-1 must match them column by column (GPU)."""
import os

import numpy as np
import pytest

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
FILE = os.path.join(HERE, "m5inv_b1.5_c0.5_M51.8_m0.002_Ls12.txt")
B_, C_, M5_, MASS, LS = 1.5, 0.5, 1.8, 0.002, 12


def load():
    rows = [l.split() for l in open(FILE) if not l.startswith("#")]
    M = np.array(rows, dtype=np.float64)
    return M[:LS], M[LS:]


def test_oracle_reproduces_stored_m5inv(orc):
    U = np.zeros((16, 4, 3, 3), dtype=np.complex128)
    for mu in range(4):
        U[:, mu] = np.eye(3)
    o = orc.Oracle((2, 2, 2, 2), LS, B_, C_, M5_, MASS, U)
    for chi, M in enumerate(load()):
        np.testing.assert_allclose(o.m5inv_closed(chi), M, rtol=1e-15, atol=1e-30)


@pytest.mark.gpu
def test_library_m5inv_matches_stored_values():
    torch = pytest.importorskip("torch")
    from paper_2104_05615_gb300 import inputs
    from paper_2104_05615_gb300.lattice import Lattice
    dims = (4, 4, 4, 4)
    lat = Lattice(dims, LS, B_, C_, M5_, MASS, inputs.gauge_field(dims, 0.3, 9))
    stored = load()
    for spin, chi in ((0, 0), (1, 0), (2, 1), (3, 1)):
        for t in (0, 5, LS - 1):
            x = torch.zeros(lat.shape, dtype=torch.complex128, device="cuda")
            x[t, 3, spin, 1] = 1.0
            y = lat.apply("m5inv", x, "f64").cpu().numpy()
            col = y[:, 3, spin, 1]
            np.testing.assert_allclose(col.real, stored[chi][:, t], rtol=1e-12, atol=1e-15)
            assert np.abs(col.imag).max() == 0.0
            y[:, 3, spin, 1] = 0
            assert np.abs(y).max() == 0.0      # diagonal in site, spin and colour
