"""GPU solves through the C ABI, checked by the FP64 CPU oracle
(arXiv:0911.3191 Sec. 5: BiCGstab and CG on the normal equations, pure FP64
and with the reliable-update mixed-precision scheme of Alg. 2).

Every solve's true residual |b - M x|/|b| is recomputed by the oracle's
operator on the host from the returned x and must be <= tol; the solution
must agree with the oracle's own FP64 solve to within the conditioning of
the system."""
import numpy as np
import pytest

import lattice_inputs as li
import oracle

pytestmark = pytest.mark.gpu

PRECS = [0, 1, 2, 3, 4]


@pytest.fixture(scope="module")
def small():
    """8^3 x 16, U = exp(0.5 i H), kappa = 0.12 (the small FP64 workload)."""
    import paper_0911_3191_gb300 as m
    dims = (8, 8, 8, 16)
    kappa = 0.12
    U = li.gauge(dims, 0.5, 1000)
    b = li.gaussian_spinor(dims, 2000)
    x_ref, st, iters, rel = oracle.solve(b, U, dims, kappa, tol=1e-12)
    assert st == 0
    wd = m.WilsonDirac(dims)
    wd.load_gauge(U)
    return m, wd, dims, kappa, U, b, x_ref, iters


@pytest.mark.parametrize("solver", [0, 1])
@pytest.mark.parametrize("prec", PRECS)
def test_solve_reaches_tolerance(small, solver, prec):
    m, wd, dims, kappa, U, b, x_ref, oracle_iters = small
    x = np.zeros_like(b)
    r = wd.solve(x, b, kappa, tol=1e-12, delta=0.1, solver=solver, inner_precision=prec)
    rel = oracle.true_residual(x, b, U, dims, kappa)
    assert r.status == 0 and rel <= 1e-12, (solver, prec, r, rel)
    assert abs(r.true_rel_residual - rel) <= 0.05 * rel + 1e-16
    assert np.linalg.norm(x - x_ref) / np.linalg.norm(x_ref) < 1e-9
    if prec != 0:
        assert r.reliable_updates >= 2
    if solver == 0:
        # reliable updates keep the mixed iteration count close to FP64 (Sec. 5.4)
        assert r.iters <= 2.0 * oracle_iters + 10


def test_graph_and_host_loop_agree_bitwise(small):
    """The CUDA-graph loop and the host loop run the same kernels in the same
    order with fixed-order reductions: identical iterates."""
    m, wd, dims, kappa, U, b, _, _ = small
    xs = []
    for g in (1, 0):
        x = np.zeros_like(b)
        r = wd.solve(x, b, kappa, tol=1e-12, solver=0, inner_precision=2, use_graph=g)
        xs.append((x, r.iters, r.reliable_updates))
    assert xs[0][1:] == xs[1][1:]
    np.testing.assert_array_equal(xs[0][0], xs[1][0])


def test_repeat_solve_is_deterministic(small):
    m, wd, dims, kappa, U, b, _, _ = small
    x1, x2 = np.zeros_like(b), np.zeros_like(b)
    wd.solve(x1, b, kappa, tol=1e-10, solver=1, inner_precision=4)
    wd.solve(x2, b, kappa, tol=1e-10, solver=1, inner_precision=4)
    np.testing.assert_array_equal(x1, x2)


def test_device_solve_matches_host_solve(small):
    m, wd, dims, kappa, U, b, _, _ = small
    x = np.zeros_like(b)
    r1 = wd.solve(x, b, kappa, tol=1e-11, inner_precision=1)
    fb = wd.upload(b, m.F64)
    fx = wd.new_field(m.F64, 2)
    r2 = wd.solve_device(fx, fb, kappa, tol=1e-11, inner_precision=1)
    assert (r1.iters, r1.reliable_updates) == (r2.iters, r2.reliable_updates)
    np.testing.assert_array_equal(wd.download(fx, m.F64), x)


@pytest.mark.parametrize("prec", [0, 2])
def test_free_field_plane_wave_solution(prec):
    """U = 1, antiperiodic t: x = (1 - kappa D(p))^{-1} b exactly."""
    import paper_0911_3191_gb300 as m
    dims = (4, 6, 8, 10)
    kappa = 0.12
    wd = m.WilsonDirac(dims, t_antiperiodic=True)
    wd.load_gauge(li.unit_gauge(dims))
    x_, y_, z_, t_ = li.coords(dims)
    p = [2 * np.pi / 4, 0.0, 2 * np.pi * 3 / 8, 5 * np.pi / 10]
    u = np.random.default_rng(2).normal(size=(4, 3)) + 0j
    b = np.exp(1j * (p[0] * x_ + p[1] * y_ + p[2] * z_ + p[3] * t_))[:, None, None] * u[None]
    G = [oracle.gamma(k) for k in range(4)]
    Dp = sum(2 * np.cos(p[k]) * np.eye(4) - 2j * np.sin(p[k]) * G[k] for k in range(4))
    want = np.einsum("ab,sbc->sac", np.linalg.inv(np.eye(4) - kappa * Dp), b)
    x = np.zeros_like(b)
    r = wd.solve(x, b, kappa, tol=1e-12, inner_precision=prec)
    assert r.status == 0
    assert np.linalg.norm(x - want) / np.linalg.norm(want) < 1e-10


def test_zero_source(small):
    m, wd, dims, kappa, U, b, _, _ = small
    x = np.ones_like(b)
    r = wd.solve(x, np.zeros_like(b), kappa, inner_precision=2)
    assert r.status == 0 and np.all(x == 0)


def test_nan_source_reports_numeric(small):
    m, wd, dims, kappa, U, b, _, _ = small
    bad = b.copy()
    bad[17, 2, 1] = np.nan
    x = np.zeros_like(b)
    r = wd.solve(x, bad, kappa, inner_precision=2, check=False)
    assert r.status == 6  # WD_ERR_NUMERIC


def test_max_iter_reports_not_converged(small):
    m, wd, dims, kappa, U, b, _, _ = small
    x = np.zeros_like(b)
    r = wd.solve(x, b, kappa, tol=1e-12, max_iter=5, inner_precision=1, check=False)
    assert r.status == 4 and r.iters >= 5
    rel = oracle.true_residual(x, b, U, dims, kappa)
    assert abs(rel - r.true_rel_residual) <= 1e-6 * rel  # x and info still written
    assert rel < 1.0


def test_invalid_arguments(small):
    m, wd, dims, kappa, U, b, _, _ = small
    x = np.zeros_like(b)
    with pytest.raises(m.WDError) as e:
        wd.solve(x, b, kappa, delta=1.5, inner_precision=2)
    assert e.value.status == 1
    with pytest.raises(m.WDError):
        wd.solve(x, b, kappa, inner_precision=9)


@pytest.mark.parametrize("solver", [0, 1])
@pytest.mark.parametrize("kappa", [0.12, 0.124])
def test_full_size_24x64_mixed_vs_fp64(solver, kappa):
    """The 24^3 x 64, eps = 0.3 workload: mixed (Q16 inner, delta = 0.1) and
    FP64 solves both reach 1e-12, checked by the oracle operator on the host."""
    import paper_0911_3191_gb300 as m
    dims = (24, 24, 24, 64)
    U = li.gauge(dims, 0.3, 1001)
    b = li.gaussian_spinor(dims, 2001)
    wd = m.WilsonDirac(dims)
    wd.load_gauge(U)
    iters = {}
    for prec in (0, 2, 1):
        x = np.zeros_like(b)
        r = wd.solve(x, b, kappa, tol=1e-12, solver=solver, inner_precision=prec)
        rel = oracle.true_residual(x, b, U, dims, kappa)
        assert r.status == 0 and rel <= 1e-12, (prec, r, rel)
        iters[prec] = r.iters
    # Sec. 5.4: reliable updates cost a modest number of extra iterations
    assert iters[2] <= 1.5 * iters[0] + 20
    wd.close()


@pytest.mark.parametrize("solver", [0, 1])
@pytest.mark.parametrize("prec,eps_in", [(2, 0.1), (2, 0.01), (1, 1e-3), (1, 1e-5)])
def test_defect_correction_alg1(small, solver, prec, eps_in):
    """Alg. 1: inner solves to eps_in with a restart at each FP64 correction;
    it reaches the FP64 tolerance like the reliable-update scheme."""
    m, wd, dims, kappa, U, b, x_ref, oracle_iters = small
    x = np.zeros_like(b)
    r = wd.solve(x, b, kappa, tol=1e-12, delta=eps_in, solver=solver, inner_precision=prec, restart=True)
    rel = oracle.true_residual(x, b, U, dims, kappa)
    assert r.status == 0 and rel <= 1e-12, (r, rel)
    assert np.linalg.norm(x - x_ref) / np.linalg.norm(x_ref) < 1e-9
    assert r.reliable_updates >= 1
    with pytest.raises(m.WDError):
        wd.solve(x, b, kappa, inner_precision=0, restart=True)


@pytest.mark.parametrize("solver", [0, 1])
@pytest.mark.parametrize("prec", [2, 3, 4])
def test_xhat_in_fp32(small, solver, prec):
    """x_hat kept in FP32 under a 16-bit inner precision (the option of
    keeping the accumulated correction above the inner precision): same
    tolerance, same solution."""
    m, wd, dims, kappa, U, b, x_ref, oracle_iters = small
    x = np.zeros_like(b)
    r = wd.solve(x, b, kappa, tol=1e-12, solver=solver, inner_precision=prec, xhat_f32=True)
    rel = oracle.true_residual(x, b, U, dims, kappa)
    assert r.status == 0 and rel <= 1e-12, (r, rel)
    assert np.linalg.norm(x - x_ref) / np.linalg.norm(x_ref) < 1e-9
    # the graph and the host loop agree bit for bit with this option too
    x2 = np.zeros_like(b)
    r2 = wd.solve(x2, b, kappa, tol=1e-12, solver=solver, inner_precision=prec, xhat_f32=True, use_graph=False)
    assert (r.iters, r.reliable_updates) == (r2.iters, r2.reliable_updates)
    np.testing.assert_array_equal(x, x2)


@pytest.mark.parametrize("solver", [0, 1])
@pytest.mark.parametrize("prec", [0, 2, 4])
def test_status_ok_implies_reported_residual_below_tol(small, solver, prec):
    """A solve that returns WD_OK reports a full FP64 true residual at or below
    tol, and the oracle agrees; any solve whose reconstructed x misses tol
    returns WD_ERR_NOT_CONVERGED instead."""
    m, wd, dims, kappa, U, b, _, _ = small
    for tol in (1e-5, 1e-7, 1e-9, 1e-11):
        x = np.zeros_like(b)
        r = wd.solve(x, b, kappa, tol=tol, delta=0.1, solver=solver, inner_precision=prec, check=False)
        rel = oracle.true_residual(x, b, U, dims, kappa)
        if r.status == 0:
            assert r.true_rel_residual <= tol and rel <= tol * (1 + 1e-6), (tol, r, rel)
        else:
            assert r.status == 4 and r.true_rel_residual > tol, (tol, r)


@pytest.mark.parametrize("prec", [0, 2, 4])
def test_initial_guess_from_a_rough_solution(small, prec):
    """initial_guess: a solve to 1e-4 followed by one to 1e-12 started from
    its x reaches the tolerance (checked by the oracle), with fewer
    iterations than from zero; the first step is the FP64 residual of the
    start (one reliable update)."""
    m, wd, dims, kappa, U, b, x_ref, _ = small
    x = np.zeros_like(b)
    r0 = wd.solve(x, b, kappa, tol=1e-12, solver=0, inner_precision=prec)
    x = np.zeros_like(b)
    rough = wd.solve(x, b, kappa, tol=1e-4, solver=0, inner_precision=prec)
    assert rough.status == 0 and oracle.true_residual(x, b, U, dims, kappa) <= 1e-4
    r = wd.solve(x, b, kappa, tol=1e-12, solver=0, inner_precision=prec, initial_guess=True)
    rel = oracle.true_residual(x, b, U, dims, kappa)
    assert r.status == 0 and rel <= 1e-12, (prec, r, rel)
    assert np.linalg.norm(x - x_ref) / np.linalg.norm(x_ref) < 1e-9
    assert r.reliable_updates >= 1
    assert r.iters < r0.iters, (r.iters, r0.iters)


def test_initial_guess_that_meets_tol_returns_at_once(small):
    """Started from a solution that already meets tol (on the device, from
    device fields), the solve runs no iteration; the returned x keeps its
    even half and gets the odd half rebuilt from it, with the same residual
    to rounding."""
    import torch
    m, wd, dims, kappa, U, b, _, _ = small
    fb = wd.upload(b, m.F64)
    fx = wd.new_field(m.F64, 2)
    r1 = wd.solve_device(fx, fb, kappa, tol=1e-10, solver=0, inner_precision=2)
    assert r1.status == 0
    before = fx.clone()
    r2 = wd.solve_device(fx, fb, kappa, tol=1e-10, solver=0, inner_precision=2, initial_guess=True)
    torch.cuda.synchronize()
    assert r2.status == 0 and r2.iters == 0 and r2.reliable_updates == 0, r2
    half = fx.numel() // 2
    assert torch.equal(fx[:half], before[:half])
    rel2 = r2.true_rel_residual
    assert rel2 <= 1e-10 and abs(rel2 - r1.true_rel_residual) <= 1e-3 * r1.true_rel_residual + 1e-15


def test_initial_guess_needs_bicgstab_with_reliable_updates(small):
    m, wd, dims, kappa, U, b, _, _ = small
    x = np.zeros_like(b)
    with pytest.raises(m.WDError):
        wd.solve(x, b, kappa, tol=1e-8, solver=1, inner_precision=2, initial_guess=True)
    with pytest.raises(m.WDError):
        wd.solve(x, b, kappa, tol=1e-8, solver=0, inner_precision=2, restart=True, initial_guess=True)
