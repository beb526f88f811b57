"""GPU solvers through the C ABI; every solution is checked with the oracle's
FP64 true residual ||b - D^+D x|| / ||b||."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2104_05615_gb300 import inputs  # noqa: E402


def make(orc, dims, Ls, sub, mass, eps, seed=5):
    from paper_2104_05615_gb300.lattice import Lattice
    U = inputs.gauge_field(dims, eps, seed)
    lat = Lattice(dims, Ls, 1.5, 0.5, 1.8, mass, U, sub)
    o = orc.Oracle(dims, Ls, 1.5, 0.5, 1.8, mass, U)
    b = inputs.gaussian_spinor_cb(dims, Ls, seed + 100)
    return lat, o, b


@pytest.mark.gpu
def test_cg_fp64_config_c1(orc):
    """4^4, Ls=8, FP64 CG to 1e-10 (the small workload); iteration count as the oracle's."""
    cfg = inputs.CONFIGS["C1"]
    from paper_2104_05615_gb300.lattice import Lattice
    U = inputs.gauge_field(cfg["dims"], cfg["eps"], cfg["gauge_seed"])
    lat = Lattice(cfg["dims"], cfg["Ls"], cfg["b"], cfg["c"], cfg["M5"], cfg["mass"], U)
    o = orc.from_config(cfg, U)
    b = inputs.gaussian_spinor_cb(cfg["dims"], cfg["Ls"], cfg["src_seed"])
    x, st = lat.solve(torch.from_numpy(b).cuda(), mspcg=False, tol=1e-10, outer_prec="f64")
    xr = x.cpu().numpy()
    assert o.true_residual(xr, b) <= 1e-10 * 1.01
    ref = o.pcg(b, tol=1e-10, maxiter=5000)
    assert abs(st["outer_iters"] - ref["iters"]) <= 2
    assert np.linalg.norm(xr - ref["x"]) / np.linalg.norm(ref["x"]) < 1e-8


@pytest.mark.gpu
def test_mixed_cg_reliable_updates(orc):
    lat, o, b = make(orc, (8, 4, 4, 4), 8, None, 0.01, 0.5)
    x, st = lat.solve(torch.from_numpy(b).cuda(), mspcg=False, tol=1e-10, outer_prec="f32")
    assert st["converged"] and st["reliable_updates"] >= 2
    assert o.true_residual(x.cpu().numpy(), b) <= 1e-10 * 1.01


@pytest.mark.gpu
@pytest.mark.parametrize("inner", ["f32", "f16", "bf16", "fx16", "fx8"])
def test_mspcg_converges_and_beats_cg(orc, inner):
    lat, o, b = make(orc, (8, 8, 4, 4), 8, (4, 4, 4, 4), 0.01, 0.5)
    bd = torch.from_numpy(b).cuda()
    x, st = lat.solve(bd, mspcg=True, tol=1e-10, inner_prec=inner, inner_iters=6)
    assert o.true_residual(x.cpu().numpy(), b) <= 1e-10 * 1.01
    _, st_cg = lat.solve(bd, mspcg=False, tol=1e-10)
    assert st["outer_iters"] < st_cg["outer_iters"]


@pytest.mark.gpu
def test_preconditioner_matches_oracle(orc):
    """z = (+)_s CG_k(A_s) r with FP32 inner storage vs the FP64 oracle."""
    from paper_2104_05615_gb300 import binding as B
    lat, o, r = make(orc, (8, 4, 4, 4), 8, (4, 4, 4, 4), 0.05, 0.5)
    rd = torch.from_numpy(r).cuda()
    z = torch.empty_like(rd)
    B.dwf_precondition(lat.h, z, rd, B.default_params(inner_prec=B.DWF_F32, inner_iters=4))
    zr = o.precond(r, k=4, sub=(4, 4, 4, 4))
    e = np.linalg.norm(z.cpu().numpy() - zr) / np.linalg.norm(zr)
    assert e < 1e-4, e


@pytest.mark.gpu
def test_reduced_ls_preconditioner_matches_oracle(orc):
    from paper_2104_05615_gb300 import binding as B
    from paper_2104_05615_gb300.lattice import heuristic_T
    lat, o, r = make(orc, (8, 4, 4, 4), 8, (4, 4, 4, 4), 0.05, 0.5)
    rng = np.random.default_rng(3)
    T = heuristic_T(8, 4) + 0.05 * (rng.standard_normal((16, 32)) + 1j * rng.standard_normal((16, 32)))
    lat.set_reduced_ls(4, T, 0.3)
    rd = torch.from_numpy(r).cuda()
    z = torch.empty_like(rd)
    B.dwf_precondition(lat.h, z, rd, B.default_params(inner_prec=B.DWF_F32, inner_iters=4,
                                                       use_reduced_ls=1))
    zr = o.precond(r, orc.PREC_REDUCED, k=4, sub=(4, 4, 4, 4), Ls_hat=4, T=T, mu=0.3)
    e = np.linalg.norm(z.cpu().numpy() - zr) / np.linalg.norm(zr)
    assert e < 1e-4, e


@pytest.mark.gpu
@pytest.mark.parametrize("inner,tol", [("bf16", 2e-2), ("fx8", 6e-2)])
def test_reduced_ls_preconditioner_tensor_core_transform(orc, inner, tol):
    """With BF16 or 8-bit inner storage the forward map r -> T r runs on the
    tensor cores with BF16 operands and FP32 accumulation (input and T
    rounded to BF16, the precision of the storage it feeds).  Against the
    FP64 oracle's reduced-Ls preconditioner with a dense T: the bound is a
    few roundings of the inner storage (BF16 2^-9, 8-bit fixed point 2^-8 of
    the site scale per element) and of T carried through two inner
    iterations, far below the O(1) error of a misplaced operand row or
    column."""
    from paper_2104_05615_gb300 import binding as B
    from paper_2104_05615_gb300.lattice import heuristic_T, PREC
    lat, o, r = make(orc, (8, 4, 4, 4), 8, (4, 4, 4, 4), 0.05, 0.5)
    rng = np.random.default_rng(4)
    T = heuristic_T(8, 4) + 0.2 * (rng.standard_normal((16, 32)) + 1j * rng.standard_normal((16, 32)))
    lat.set_reduced_ls(4, T, 0.3)
    rd = torch.from_numpy(r).cuda()
    z = torch.empty_like(rd)
    B.dwf_precondition(lat.h, z, rd, B.default_params(inner_prec=PREC[inner], inner_iters=2,
                                                       use_reduced_ls=1))
    zr = o.precond(r, orc.PREC_REDUCED, k=2, sub=(4, 4, 4, 4), Ls_hat=4, T=T, mu=0.3)
    e = np.linalg.norm(z.cpu().numpy() - zr) / np.linalg.norm(zr)
    assert e < tol, e


@pytest.mark.gpu
@pytest.mark.parametrize("inner", ["bf16", "fx16", "fx8"])
def test_mspcg_reduced_ls_converges(orc, inner):
    from paper_2104_05615_gb300.lattice import heuristic_T
    lat, o, b = make(orc, (8, 8, 4, 4), 8, (4, 4, 4, 4), 0.01, 0.5)
    lat.set_reduced_ls(4, heuristic_T(8, 4), 0.85)
    x, st = lat.solve(torch.from_numpy(b).cuda(), mspcg=True, tol=1e-10, inner_prec=inner,
                      use_reduced_ls=1)
    assert o.true_residual(x.cpu().numpy(), b) <= 1e-10 * 1.01


@pytest.mark.gpu
@pytest.mark.parametrize("inner", ["f16", "fx16"])
def test_batched_mspcg_uneven_systems(orc, inner):
    """Independent lattices of different sizes and masses in one batch; each
    system's answer verified by its own oracle."""
    from paper_2104_05615_gb300 import binding as B
    from paper_2104_05615_gb300.lattice import Lattice
    shapes = [((8, 8, 8, 8), 0.004), ((8, 8, 8, 12), 0.01), ((12, 8, 8, 8), 0.02)]
    lats, oracles, bs, xs = [], [], [], []
    for k, (dims, m) in enumerate(shapes):
        U = inputs.gauge_field(dims, 0.5, 300 + k)
        lats.append(Lattice(dims, 4, 1.5, 0.5, 1.8, m, U, (4, 4, 4, 4)))
        oracles.append(orc.Oracle(dims, 4, 1.5, 0.5, 1.8, m, U))
        b = inputs.gaussian_spinor_cb(dims, 4, 400 + k)
        bs.append(b)
        xs.append(torch.zeros(b.shape, dtype=torch.complex128, device="cuda"))
    bt = B.dwf_batch_create([l.h for l in lats])
    try:
        bd = [torch.from_numpy(b).cuda() for b in bs]
        from paper_2104_05615_gb300.lattice import PREC
        tot, per = B.dwf_batch_mspcg(bt, xs, bd, B.default_params(tol=1e-9, inner_prec=PREC[inner]))
        assert tot.converged
        for k in range(3):
            assert oracles[k].true_residual(xs[k].cpu().numpy(), bs[k]) <= 1e-9 * 1.01
    finally:
        B.dwf_batch_destroy(bt)


@pytest.mark.gpu
def test_solve_host_buffers(orc):
    from paper_2104_05615_gb300 import binding as B
    lat, o, b = make(orc, (8, 4, 4, 4), 8, (4, 4, 4, 4), 0.05, 0.5)
    x = np.zeros_like(b)
    st = B.dwf_solve_host(lat.h, x, b, B.default_params(tol=1e-10), use_mspcg=True)
    assert st.converged
    assert o.true_residual(x, b) <= 1e-10 * 1.01


@pytest.mark.gpu
def test_noconvergence_reports_status(orc):
    from paper_2104_05615_gb300 import binding as B
    lat, o, b = make(orc, (8, 4, 4, 4), 8, (4, 4, 4, 4), 0.01, 0.5)
    bd = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bd)
    st = B.dwf_cg(lat.h, x, bd, B.default_params(tol=1e-10, maxiter=5), raise_on_noconv=False)
    assert not st.converged and st.outer_iters == 5
    # x holds the last iterate: a better residual than x = 0
    assert o.true_residual(x.cpu().numpy(), b) < 1.0


@pytest.mark.gpu
def test_graph_captured_solve_matches_direct_launches(orc):
    """The outer iteration replayed as CUDA graphs gives the same iterates as
    launching every kernel directly."""
    lat, o, b = make(orc, (8, 8, 4, 4), 8, (4, 4, 4, 4), 0.01, 0.5)
    bd = torch.from_numpy(b).cuda()
    lat.solve(bd, mspcg=True, tol=1e-10, inner_prec="f16", use_graph=0)  # tunes launch shapes
    x1, s1 = lat.solve(bd, mspcg=True, tol=1e-10, inner_prec="f16", use_graph=1)
    x0, s0 = lat.solve(bd, mspcg=True, tol=1e-10, inner_prec="f16", use_graph=0)
    assert s1["outer_iters"] == s0["outer_iters"]
    assert torch.equal(x1, x0)
    assert s1["kernel_launches"] == s0["kernel_launches"]


@pytest.mark.gpu
@pytest.mark.parametrize("graph", [0, 1])
def test_live_operator_timing(orc, graph):
    """time_kernels: every outer D^+D and every inner local operator of the
    solve is timed with events on the solve's stream, in graphs too."""
    from paper_2104_05615_gb300 import binding as B
    lat, o, b = make(orc, (8, 8, 4, 4), 8, (4, 4, 4, 4), 0.01, 0.5)
    bd = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bd)
    st = B.dwf_mspcg(lat.h, x, bd, B.default_params(tol=1e-10, inner_prec=B.DWF_F16, inner_iters=6,
                                                    use_graph=graph, time_kernels=1))
    assert st.converged
    assert st.outer_op_count == st.outer_iters
    # one preconditioner before the loop and one per iteration that continues
    assert st.local_op_count == st.inner_iters_total
    assert st.inner_iters_total >= 6 * st.outer_iters - 6
    assert 0 < st.outer_op_ms / st.outer_op_count < 50
    assert 0 < st.local_op_ms / st.local_op_count < 50
    assert st.local_op_ms < st.time_total_ms


@pytest.mark.gpu
@pytest.mark.parametrize("outer", ["f16", "bf16", "fx16"])
@pytest.mark.parametrize("mspcg", [True, False])
def test_16bit_outer_iterations(orc, outer, mspcg):
    """16-bit outer vectors (Sec. 3.2: 16-bit outer iterations with FP64
    reliable updates) reach the FP64 tolerance."""
    lat, o, b = make(orc, (8, 8, 4, 4), 8, (4, 4, 4, 4), 0.01, 0.5)
    x, st = lat.solve(torch.from_numpy(b).cuda(), mspcg=mspcg, tol=1e-10, outer_prec=outer,
                      inner_prec="f16", maxiter=20000)
    assert st["converged"] and st["reliable_updates"] >= 1
    assert o.true_residual(x.cpu().numpy(), b) <= 1e-10 * 1.01


@pytest.mark.gpu
@pytest.mark.parametrize("mspcg", [True, False])
def test_check_every_skips_host_reads(orc, mspcg):
    """check_every = 4: the host reads the residual (and decides reliable updates
    and convergence) every fourth iteration only; the solve still reaches the
    oracle-verified tol, with at most the 3 iterations a check can lag plus one."""
    lat, o, b = make(orc, (8, 8, 4, 4), 8, (4, 4, 4, 4), 0.01, 0.5)
    bd = torch.from_numpy(b).cuda()
    kw = dict(mspcg=mspcg, tol=1e-10, inner_prec="f16", inner_iters=6)
    _, st1 = lat.solve(bd, **kw)
    x4, st4 = lat.solve(bd, check_every=4, **kw)
    assert st4["converged"] and o.true_residual(x4.cpu().numpy(), b) <= 1e-10 * 1.01
    assert st4["outer_iters"] % 4 == 0  # convergence is seen at check points only
    assert st4["outer_iters"] <= st1["outer_iters"] + 4
