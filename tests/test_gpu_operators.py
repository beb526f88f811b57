"""GPU operator parity against the FP64 oracle, through the C ABI.

Relative error ||out - out_oracle|| / ||out_oracle|| bounds (the accuracy each
storage format allows): FP64 1e-12, FP32 1e-6, FP16/BF16 and 16-bit fixed
point 5e-3.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2104_05615_gb300 import inputs  # noqa: E402

# 8-bit fixed point: every stored component is off by at most half of
# max|colour-spinor| / 127, an RMS relative error of about 2.5 / (127 sqrt(12))
# = 5.7e-3 for a Gaussian colour-spinor (its max is ~2.5 x its RMS); the four
# rounded stage outputs of D^+D add in quadrature to ~1.1e-2, bounded here by
# 3e-2 (the input rounding is common to both sides)
TOL = {"f64": 1e-12, "f32": 1e-6, "f16": 5e-3, "bf16": 5e-3, "fx16": 5e-3, "fx8": 3e-2}

CASES = {
    # name: dims, Ls, sub, mass, eps, antiperiodic
    "part_x": ((8, 4, 4, 4), 8, (4, 4, 4, 4), 0.05, 0.5, 0),
    "ragged": ((6, 2, 2, 2), 4, None, 0.1, 0.6, 0),
    "ragged_part": ((12, 2, 2, 2), 4, (6, 2, 2, 2), 0.02, 0.6, 0),
    "antiperiodic": ((4, 4, 4, 6), 6, None, 0.03, 0.4, 1),
    "ls12": ((4, 4, 4, 8), 12, (4, 4, 4, 4), 0.01, 0.5, 0),
    "ls16_4d": ((8, 8, 4, 4), 16, (4, 4, 4, 4), 0.002, 0.6, 0),
}


def relerr(a, b):
    return np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel())


def setup_case(orc, name):
    from paper_2104_05615_gb300.lattice import Lattice
    dims, Ls, sub, mass, eps, anti = CASES[name]
    U = inputs.gauge_field(dims, eps, 17)
    lat = Lattice(dims, Ls, 1.5, 0.5, 1.8, mass, U, sub, anti)
    o = orc.Oracle(dims, Ls, 1.5, 0.5, 1.8, mass, U, anti)
    x = inputs.gaussian_spinor_cb(dims, Ls, 99)
    return lat, o, x, (sub or dims)


@pytest.mark.gpu
@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("prec", ["f64", "f32", "f16", "bf16", "fx16", "fx8"])
def test_operator_parity(orc, name, prec):
    from paper_2104_05615_gb300.lattice import to_device, to_numpy
    lat, o, x, sub = setup_case(orc, name)
    xd = to_device(x, prec)
    xin = to_numpy(xd)  # the rounded input both sides see
    ref = {"D": o.D(xin), "Ddag": o.D(xin, dagger=True), "DdagD": o.DdagD(xin),
           "local": o.local_DdagD(xin, sub),
           "m5inv": o.apply5(o.matrix5(3), xin), "m5invdag": o.apply5(o.matrix5(3, True), xin)}
    for op, want in ref.items():
        got = to_numpy(lat.apply(op, xd, prec))
        e = relerr(got, want)
        assert e < TOL[prec], f"{name} {prec} {op}: relative error {e:.3e}"


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["f64", "f32", "f16", "bf16", "fx16", "fx8"])
def test_pack_roundtrip(orc, prec):
    from paper_2104_05615_gb300.lattice import to_device, to_numpy
    lat, o, x, sub = setup_case(orc, "ragged_part")
    xd = to_device(x, prec)
    p = lat.pack(xd, prec)
    back = lat.unpack(p, prec)
    if prec in ("f64", "f32"):
        assert torch.equal(back, xd)
    elif prec == "fx16":
        assert torch.equal(back.cpu(), fixed16_roundtrip(xd.cpu()))
    elif prec == "fx8":
        assert torch.equal(back.cpu(), fixed_roundtrip(xd.cpu(), 127))
    else:  # FP16 packs with one scale per colour-spinor
        assert relerr(to_numpy(back), to_numpy(xd)) < 2e-3


def fixed16_roundtrip(x):
    return fixed_roundtrip(x, 32767)


def fixed_roundtrip(x, limit):
    """The fixed-point formats of Sec. 3.2 written out (integer-limit 32767 for
    16 bits, 127 for 8 bits): per colour-spinor (24 FP32 reals) m = max |v|,
    inv = limit / m in FP32, q = rint(v * inv) of the exact product (ties to
    even), and the value read back is q * (m / limit) in FP32 (m = 0: all
    zero)."""
    v = torch.view_as_real(x).reshape(x.shape[0], x.shape[1], 24).numpy()
    m = np.abs(v).max(axis=2, keepdims=True).astype(np.float32)
    lim = np.float32(limit)
    with np.errstate(divide="ignore"):
        inv = np.where(m > 0, lim / m, np.float32(0)).astype(np.float32)
    sc = np.where(m > 0, m / lim, np.float32(1)).astype(np.float32)
    q = np.rint(v.astype(np.float64) * inv.astype(np.float64))  # FP32 x FP32 is exact in FP64
    assert np.abs(q).max() <= limit
    q = q.astype(np.float32)
    back = (q * sc).astype(np.float32).reshape(x.shape + (2,))
    return torch.view_as_complex(torch.from_numpy(np.ascontiguousarray(back)))


@pytest.mark.gpu
def test_apply_packed_matches_canonical(orc):
    from paper_2104_05615_gb300 import binding as B
    from paper_2104_05615_gb300.lattice import to_device
    lat, o, x, sub = setup_case(orc, "part_x")
    xd = to_device(x, "f32")
    p_in = lat.pack(xd, "f32")
    p_out = lat.packed("f32")
    B.dwf_apply_packed(lat.h, p_out, p_in, B.DWF_OP_DDAGD, B.DWF_F32)
    a = lat.unpack(p_out, "f32")
    b = lat.apply("DdagD", xd, "f32")
    assert torch.equal(a, b)


@pytest.mark.gpu
def test_operator_deterministic(orc):
    lat, o, x, sub = setup_case(orc, "ls12")
    from paper_2104_05615_gb300.lattice import to_device
    xd = to_device(x, "f32")
    a = lat.apply("DdagD", xd, "f32")
    b = lat.apply("DdagD", xd, "f32")
    assert torch.equal(a, b)


@pytest.mark.gpu
def test_invalid_arguments_rejected():
    from paper_2104_05615_gb300 import binding as B
    U = inputs.gauge_field((4, 4, 4, 4), 0.1, 1)
    with pytest.raises(B.DwfError):   # odd extent
        B.dwf_create(U, (3, 4, 4, 4), 8, 1.5, 0.5, 1.8, 0.1)
    with pytest.raises(B.DwfError):   # block too large for the snake halo
        B.dwf_create(U, (4, 4, 4, 4), 8, 1.5, 0.5, 1.8, 0.1, (2, 4, 4, 4))
    with pytest.raises(B.DwfError):   # block does not divide
        B.dwf_create(U, (4, 4, 4, 4), 8, 1.5, 0.5, 1.8, 0.1, (6, 4, 4, 4))


@pytest.mark.gpu
@pytest.mark.parametrize("name", ["part_x", "ragged_part", "ls16_4d"])
@pytest.mark.parametrize("prec", ["f32", "f16"])
def test_truncated_local_operator(orc, name, prec):
    """dwf_set_local_truncated: the local operator with Dirichlet walls on every
    hop (the left side of Eq. (eq:diri)) against the oracle's truncated
    product; switching back gives R_s D^+D R_s^T again."""
    from paper_2104_05615_gb300 import binding as B
    from paper_2104_05615_gb300.lattice import to_device, to_numpy
    lat, o, x, sub = setup_case(orc, name)
    xd = to_device(x, prec)
    xin = to_numpy(xd)
    want_t = o.local_DdagD_truncated(xin, sub)
    want_s = o.local_DdagD(xin, sub)
    assert relerr(want_t, want_s) > 1e-3  # the snake terms matter here
    B.dwf_set_local_truncated(lat.h, 1)
    e = relerr(to_numpy(lat.apply("local", xd, prec)), want_t)
    assert e < TOL[prec], f"truncated {name} {prec}: {e:.3e}"
    B.dwf_set_local_truncated(lat.h, 0)
    e = relerr(to_numpy(lat.apply("local", xd, prec)), want_s)
    assert e < TOL[prec], f"snake {name} {prec}: {e:.3e}"


@pytest.mark.gpu
def test_long_fifth_dimension_runtime_path(orc):
    """Ls = 20 (no compile-time instance): FP32 / FP64 operators against the
    oracle; the 16-bit tensor-core stages need Ls <= 16 and say so."""
    from paper_2104_05615_gb300 import binding as B
    from paper_2104_05615_gb300.lattice import Lattice, to_device, to_numpy
    dims, Ls, sub = (8, 4, 4, 4), 20, (4, 4, 4, 4)
    U = inputs.gauge_field(dims, 0.5, 8)
    lat = Lattice(dims, Ls, 1.5, 0.5, 1.8, 0.02, U, sub)
    o = orc.Oracle(dims, Ls, 1.5, 0.5, 1.8, 0.02, U)
    x = inputs.gaussian_spinor_cb(dims, Ls, 77)
    for prec in ("f64", "f32"):
        xd = to_device(x, prec)
        xin = to_numpy(xd)
        for op, want in (("DdagD", o.DdagD(xin)), ("local", o.local_DdagD(xin, sub))):
            e = relerr(to_numpy(lat.apply(op, xd, prec)), want)
            assert e < TOL[prec], (prec, op, e)
    with pytest.raises(B.DwfError):
        lat.apply("DdagD", to_device(x, "f16"), "f16")


@pytest.mark.gpu
def test_kernel_config_validation(orc):
    from paper_2104_05615_gb300 import binding as B
    lat, o, x, sub = setup_case(orc, "part_x")
    for tile, gather in ((6, 0), (3, 0), (8, 2), (0, 0)):
        with pytest.raises(B.DwfError) as e:
            B.dwf_set_kernel_config(lat.h, B.DWF_F32, 0, tile, gather)
        assert e.value.status == B.DWF_EINVAL
    B.dwf_set_kernel_config(lat.h, B.DWF_F32, 0, 8, 0)
    c = B.dwf_kernel_config()
    B.check(B.lib().dwf_get_kernel_config(lat.h, B.DWF_F32, 0, B.C.byref(c)), lat.h)
    assert (c.tile_sites, c.gather) == (8, 0)


@pytest.mark.gpu
def test_fma_peak_measured(orc):
    """dwf_fma_peak: a plausible FP32 and FP64 FMA rate, FP64 below FP32, and
    storage formats without CUDA-core arithmetic of their own rejected."""
    from paper_2104_05615_gb300 import binding as B
    lat, o, x, sub = setup_case(orc, "ragged")
    f32 = B.dwf_fma_peak(lat.h, B.DWF_F32)
    f64 = B.dwf_fma_peak(lat.h, B.DWF_F64)
    assert 1.0 < f32 < 1000.0
    assert 0.01 < f64 < f32
    for bad in (B.DWF_F16, B.DWF_BF16, B.DWF_FX16, 7):
        with pytest.raises(B.DwfError):
            B.dwf_fma_peak(lat.h, bad)


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["f64", "f32", "f16", "bf16", "fx16", "fx8"])
def test_every_kernel_config_matches_oracle(orc, prec):
    """Every launch shape the autotuner may pick (site tile x direct or
    bulk-copy neighbour gather) gives the global D^+D and the local operator
    within the format's tolerance; shapes that do not fit are refused."""
    from paper_2104_05615_gb300 import binding as B
    from paper_2104_05615_gb300.lattice import PREC, to_device, to_numpy
    lat, o, x, sub = setup_case(orc, "ls12")
    xd = to_device(x, prec)
    xin = to_numpy(xd)
    want = {"DdagD": o.DdagD(xin), "local": o.local_DdagD(xin, sub)}
    ran = set()
    for gather in (0, 1, 2):
        for tile in (4, 8, 16, 32):
            for kind, op in ((0, "DdagD"), (1, "local")):
                try:
                    B.dwf_set_kernel_config(lat.h, PREC[prec], kind, tile, gather)
                except B.DwfError as err:
                    assert err.status == B.DWF_EINVAL
                    continue
                e = relerr(to_numpy(lat.apply(op, xd, prec)), want[op])
                assert e < TOL[prec], f"{prec} {op} tile {tile} gather {gather}: {e:.3e}"
                ran.add((op, gather))
    assert {("DdagD", 0), ("local", 0)} <= ran
    if prec not in ("f64", "fx8"):
        assert {("DdagD", 1), ("local", 1)} <= ran
    if prec in ("f16", "bf16", "fx16"):
        assert {("DdagD", 2), ("local", 2)} <= ran


@pytest.mark.gpu
@pytest.mark.parametrize("name", [n for n, c in CASES.items() if c[1] % 4 == 0])
@pytest.mark.parametrize("prec", ["f16", "bf16", "fx16"])
def test_tensor_core_hop_parity(orc, name, prec):
    """The hop on the tensor cores (gather 2: projected neighbour spinors x
    links as FP16 mma with FP32 accumulation) for D, D^+, D^+D and the local
    operator against the oracle, on every lattice whose Ls it takes."""
    from paper_2104_05615_gb300 import binding as B
    from paper_2104_05615_gb300.lattice import PREC, to_device, to_numpy
    lat, o, x, sub = setup_case(orc, name)
    for kind in (0, 1):
        B.dwf_set_kernel_config(lat.h, PREC[prec], kind, 8, 2)
    xd = to_device(x, prec)
    xin = to_numpy(xd)
    ref = {"D": o.D(xin), "Ddag": o.D(xin, dagger=True), "DdagD": o.DdagD(xin),
           "local": o.local_DdagD(xin, sub)}
    for op, want in ref.items():
        e = relerr(to_numpy(lat.apply(op, xd, prec)), want)
        assert e < TOL[prec], f"{name} {prec} {op}: relative error {e:.3e}"
    assert B.dwf_get_kernel_config(lat.h, PREC[prec], 1)["gather"] == 2
