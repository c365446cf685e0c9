"""Multi-shift solves over kappa (wd_solve_multishift): one shared FP32
multi-shift BiCGstab for the shifted family M_hat(kappa_k) ~ M_hat(kappa_s) +
tau_k, then a reliable-update refinement per kappa.  Every solution is checked
against its definition: the FP64 oracle's true residual of M_kappa x = b and
the oracle's own solve of each system."""
import numpy as np
import pytest

import lattice_inputs as li
import oracle

pytestmark = pytest.mark.gpu

KAPPAS = [0.118, 0.124, 0.11, 0.12]


def setup(dims, tfix=False, anti=False, seed=1500, eps=0.5):
    import paper_0911_3191_gb300 as m
    U = li.gauge(dims, eps, seed)
    wd = m.WilsonDirac(dims, t_antiperiodic=anti)
    wd.load_gauge(U, recon=18, temporal_gauge=tfix)
    return m, wd, U


@pytest.mark.parametrize("inner", [1, 2, 3])
def test_gaussian_source_every_kappa(inner):
    """A Gaussian source (b_o != 0: two shifted families)."""
    dims = (8, 8, 8, 16)
    m, wd, U = setup(dims)
    b = li.gaussian_spinor(dims, 2500)
    xs = [np.zeros_like(b) for _ in KAPPAS]
    infos = wd.solve_multishift(xs, b, KAPPAS, tol=1e-12, inner_precision=inner)
    for x, k, info in zip(xs, KAPPAS, infos):
        rel = oracle.true_residual(x, b, U, dims, k)
        assert info.status == 0 and rel <= 1e-12, (k, info, rel)
        assert abs(info.true_rel_residual - rel) <= 0.05 * rel + 1e-15
        x_ref, st, _, _ = oracle.solve(b, U, dims, k, tol=1e-12)
        assert np.linalg.norm(x - x_ref) / np.linalg.norm(x_ref) < 1e-9, k


def test_point_source_temporal_gauge_antiperiodic():
    """An even-site point source (b_o = 0: one family), temporal gauge,
    antiperiodic time direction."""
    dims = (8, 6, 4, 16)
    m, wd, U = setup(dims, tfix=True, anti=True, seed=1501)
    b = li.point_source(dims, (0, 0, 0, 0), 1, 2)
    xs = [np.zeros_like(b) for _ in KAPPAS]
    infos = wd.solve_multishift(xs, b, KAPPAS, tol=1e-10, inner_precision=m.Q16)
    for x, k, info in zip(xs, KAPPAS, infos):
        rel = oracle.true_residual(x, b, U, dims, k, tbc_anti=True)
        assert info.status == 0 and rel <= 1e-10, (k, info, rel)


def test_loose_tol():
    """A tol above the FP32 stage target (the stage stops at tol)."""
    dims = (8, 8, 8, 16)
    m, wd, U = setup(dims, seed=1502)
    b = li.gaussian_spinor(dims, 2501)
    xs = [np.zeros_like(b) for _ in KAPPAS]
    infos = wd.solve_multishift(xs, b, KAPPAS, tol=1e-4, inner_precision=m.Q16)
    for x, k, info in zip(xs, KAPPAS, infos):
        rel = oracle.true_residual(x, b, U, dims, k)
        assert info.status == 0 and rel <= 1e-4, (k, info, rel)


def test_single_kappa_and_duplicates():
    dims = (4, 6, 8, 10)
    m, wd, U = setup(dims, seed=1503)
    b = li.gaussian_spinor(dims, 2502)
    for ks in ([0.121], [0.12, 0.12, 0.115]):
        xs = [np.zeros_like(b) for _ in ks]
        infos = wd.solve_multishift(xs, b, ks, tol=1e-12, inner_precision=m.Q16)
        for x, k, info in zip(xs, ks, infos):
            rel = oracle.true_residual(x, b, U, dims, k)
            assert info.status == 0 and rel <= 1e-12, (ks, info, rel)


def test_zero_source_and_bad_args():
    import paper_0911_3191_gb300 as m
    dims = (4, 4, 4, 8)
    _, wd, U = setup(dims, seed=1504)
    b = np.zeros((li.volume(dims), 4, 3), dtype=np.complex128)
    xs = [np.ones_like(b) for _ in range(2)]
    infos = wd.solve_multishift(xs, b, [0.12, 0.11], tol=1e-12, inner_precision=m.Q16)
    for x, info in zip(xs, infos):
        assert info.status == 0 and not np.any(x)
    b = li.gaussian_spinor(dims, 2503)
    for ks in ([], [0.1] * 33, [0.12, -0.1]):
        with pytest.raises(m.WDError):
            wd.solve_multishift([np.zeros_like(b) for _ in ks], b, ks)
