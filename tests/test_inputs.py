"""The seeded input generators (shared by the CUDA path's tests, the oracle's
tests and the bench): the counter-based SplitMix64 against the sequential
generator of its publication written with Python integers, the distributions
it feeds, the SU(3) gauge field and the workload recipes."""
import numpy as np
import pytest

from paper_2104_05615_gb300 import inputs

MASK = (1 << 64) - 1
GOLDEN = 0x9E3779B97F4A7C15


def mix64_int(z):
    """The SplitMix64 output function (Steele, Lea, Flood 2014) on a Python int."""
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
    return z ^ (z >> 31)


def sequential_splitmix(state, n):
    """The published sequential form: state += GOLDEN, output mix64(state)."""
    out = []
    for _ in range(n):
        state = (state + GOLDEN) & MASK
        out.append(mix64_int(state))
    return out


@pytest.mark.parametrize("seed,stream", [(0, 0), (103, 0), (2**40 + 7, 3), (1, 7)])
def test_counter_splitmix_is_the_sequential_generator(seed, stream):
    key = mix64_int(((seed ^ (stream << 32)) & MASK) ^ GOLDEN)
    want = sequential_splitmix(key, 64)
    got = inputs.splitmix64(seed, stream, 64)
    assert [int(v) for v in got] == want
    # counter offsets address the same sequence
    assert [int(v) for v in inputs.splitmix64(seed, stream, 8, offset=20)] == want[20:28]


def test_streams_and_seeds_differ():
    a = inputs.splitmix64(5, 0, 1000)
    assert len(set(a.tolist())) == 1000
    assert not np.intersect1d(a, inputs.splitmix64(5, 1, 1000)).size
    assert not np.intersect1d(a, inputs.splitmix64(6, 0, 1000)).size


def test_uniform_and_normal_moments():
    n = 1 << 20
    u = inputs.uniform(11, 0, n)
    assert u.min() > 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 5 * np.sqrt(1 / 12 / n)
    assert abs(u.var() - 1 / 12) < 5 * np.sqrt(1 / 180 / n)
    g = inputs.normal(12, 0, n)
    assert abs(g.mean()) < 5 / np.sqrt(n)
    assert abs(g.var() - 1.0) < 5 * np.sqrt(2 / n)
    # fourth moment of N(0,1) is 3
    assert abs(np.mean(g**4) - 3.0) < 5 * np.sqrt(96 / n)
    # odd length: the prefix of the even-length draw
    np.testing.assert_array_equal(inputs.normal(12, 0, 9), g[:9])


def test_gell_mann_normalisation():
    lam = inputs.gell_mann()
    for a in range(8):
        np.testing.assert_allclose(lam[a], lam[a].conj().T, atol=0)
        assert abs(np.trace(lam[a])) < 1e-15
        for b in range(8):
            assert abs(np.trace(lam[a] @ lam[b]) - 2.0 * (a == b)) < 1e-14


def test_gauge_links_are_su3_and_eps_sets_the_spread():
    U = inputs.gauge_field((2, 2, 2, 4), 0.6, 7).reshape(-1, 3, 3)
    eye = np.eye(3)
    assert np.abs(U @ np.conj(np.swapaxes(U, -1, -2)) - eye).max() < 1e-14
    assert np.abs(np.linalg.det(U) - 1.0).max() < 1e-14
    # eps = 0: the unit field
    U0 = inputs.gauge_field((2, 2, 2, 2), 0.0, 7)
    np.testing.assert_allclose(U0, np.broadcast_to(eye, U0.shape), atol=1e-15)
    # small eps: U = 1 + i eps H + O(eps^2) with H the seeded traceless Hermitian matrix
    e = 1e-6
    Ue = inputs.su3_exp_field(16, e, 9)
    H = np.einsum("na,aij->nij", inputs.normal(9, 0, 8 * 16).reshape(16, 8), inputs.gell_mann()) / 2
    np.testing.assert_allclose((Ue - eye) / (1j * e), H, atol=1e-5)


def test_plaquette_fingerprint():
    dims = (4, 4, 4, 4)
    assert abs(inputs.plaquette(inputs.gauge_field(dims, 0.0, 1), dims) - 1.0) < 1e-14
    p = [inputs.plaquette(inputs.gauge_field(dims, eps, 1), dims) for eps in (0.2, 0.5, 0.9)]
    assert 1.0 > p[0] > p[1] > p[2] > 0.0
    # a random gauge transformation leaves it unchanged
    U = inputs.gauge_field(dims, 0.5, 2)
    V = int(np.prod(dims))
    g = inputs.random_su3(V, 3)
    Lx, Ly, Lz, Lt = dims
    lex = np.arange(V)
    x, y, z, t = lex % Lx, (lex // Lx) % Ly, (lex // (Lx * Ly)) % Lz, lex // (Lx * Ly * Lz)
    Ug = np.empty_like(U)
    for mu, (dx, dy, dz, dt) in enumerate(((1, 0, 0, 0), (0, 1, 0, 0), (0, 0, 1, 0), (0, 0, 0, 1))):
        nb = ((x + dx) % Lx) + Lx * (((y + dy) % Ly) + Ly * (((z + dz) % Lz) + Lz * ((t + dt) % Lt)))
        Ug[:, mu] = g @ U[:, mu] @ np.conj(np.swapaxes(g[nb], -1, -2))
    assert abs(inputs.plaquette(Ug, dims) - inputs.plaquette(U, dims)) < 1e-13


def test_spinor_layouts():
    dims, Ls = (4, 2, 2, 2), 3
    x = inputs.gaussian_spinor_cb(dims, Ls, 5)
    assert x.shape == (Ls, 16, 4, 3) and x.dtype == np.complex128
    f = inputs.gaussian_spinor_full(dims, Ls, 5)
    assert f.shape == (Ls, 32, 4, 3)
    # the even/odd field is the prefix of the same stream (same seed and stream)
    np.testing.assert_array_equal(x.reshape(-1), f.reshape(-1)[:x.size])
    y = inputs.gaussian_spinor_cb(dims, Ls, 5, stream=1)
    assert abs(np.vdot(x, y)) < 5 * np.sqrt(x.size) * 2


def test_workload_recipes():
    c3 = inputs.CONFIGS["C3"]
    assert c3["dims"] == (16, 16, 16, 32) and c3["Ls"] == 12 and c3["sub"] == (8, 8, 8, 8)
    assert np.prod(c3["dims"]) // np.prod(c3["sub"]) == 32  # 32 blocks of 8^4
    for c in inputs.CONFIGS.values():
        assert all(d % s == 0 and s % 2 == 0 for d, s in zip(c["dims"], c["sub"]))
    sy = inputs.c5_systems()
    assert len(sy) == 48
    assert [s["dims"] for s in sy].count((12, 12, 12, 12)) == 16
    m = np.array([s["mass"] for s in sy])
    assert m.min() >= 0.002 and m.max() <= 0.02 and len(set(m.tolist())) == 48
    assert sum(np.prod(s["dims"]) // 2 * s["Ls"] for s in sy) == 3170304
