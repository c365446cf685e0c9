"""8-number link storage (arXiv:0911.3191 App. A.2) for the FP32 and 16-bit
copies (wd_load_gauge_opt with WD_GAUGE_RECON8), alone and with the temporal
gauge (Sec. 4.3): dslash, M_hat, batched dslash and solves against the FP64
oracle on the FP64 links; the singular links (|a1| = 1) are refused."""
import numpy as np
import pytest

import lattice_inputs as li
import oracle
from tests.wd_testutil import TOL, parity_mask, rel_err

pytestmark = pytest.mark.gpu

PRECS = [1, 2, 3, 4]


def load(dims, tfix, anti=False, seed=1300, eps=0.5):
    import paper_0911_3191_gb300 as m
    U = li.gauge(dims, eps, seed)
    wd = m.WilsonDirac(dims, t_antiperiodic=anti)
    wd.load_gauge(U, recon=18, temporal_gauge=tfix, recon8=True)
    return m, wd, U


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("tfix", [False, True])
@pytest.mark.parametrize("anti", [False, True])
@pytest.mark.parametrize("dagger", [False, True])
def test_dslash_matches_oracle(prec, tfix, anti, dagger):
    dims = (8, 6, 4, 16)
    m, wd, U = load(dims, tfix, anti, seed=1300 + prec)
    psi = li.gaussian_spinor(dims, 3700 + prec)
    for out_parity in (0, 1):
        fin = wd.upload(psi, prec, parity=1 - out_parity)
        fout = wd.new_field(prec)
        wd.dslash(fout, fin, out_parity, dagger, prec)
        got = wd.download(fout, prec, parity=out_parity)
        want = oracle.dslash(psi * parity_mask(dims, 1 - out_parity), U, dims, dagger=dagger,
                             out_parity=out_parity, tbc_anti=anti)
        assert rel_err(got, want) <= TOL[prec], (prec, tfix, anti, dagger, out_parity, rel_err(got, want))


@pytest.mark.parametrize("eps", [0.2, 3.0])
def test_f32_accuracy_weak_and_strong_fields(eps):
    """FP32 8-number links keep the FP32 dslash bar on near-unit and on
    random links (1/N amplifies rounding where |a1| is close to 1)."""
    dims = (4, 6, 8, 10)
    m, wd, U = load(dims, False, eps=eps, seed=1310)
    psi = li.gaussian_spinor(dims, 3710)
    fin = wd.upload(psi, m.F32, parity=1)
    fout = wd.new_field(m.F32)
    wd.dslash(fout, fin, 0, False, m.F32)
    got = wd.download(fout, m.F32, parity=0)
    want = oracle.dslash(psi * parity_mask(dims, 1), U, dims, out_parity=0)
    assert rel_err(got, want) <= TOL[1]


@pytest.mark.parametrize("prec", [2, 4])
def test_mhat_and_batch(prec):
    dims = (8, 6, 4, 16)
    m, wd, U = load(dims, True, anti=True)
    kappa = 0.124
    psi = li.gaussian_spinor(dims, 3720)
    fe = wd.upload(psi, prec, parity=0)
    fo = wd.new_field(prec)
    wd.apply_M(fo, fe, kappa, m.M_SCHUR_EVEN, False, prec)
    want = oracle.apply_Mhat(psi * parity_mask(dims, 0), U, dims, kappa, tbc_anti=True)
    assert rel_err(wd.download(fo, prec, parity=0), want) <= TOL[prec]
    nrhs = 3
    fb = wd.field_bytes(prec)
    srcs = [li.gaussian_spinor(dims, 3730 + r) for r in range(nrhs)]
    fin = wd.new_field(prec, nrhs)
    for r, s in enumerate(srcs):
        wd.field_import(fin[r * fb:(r + 1) * fb], s, m.EVEN, prec)
    fout = wd.new_field(prec, nrhs)
    wd.dslash_batch(fout, fin, nrhs, m.ODD, True, prec)
    for r, s in enumerate(srcs):
        got = wd.download(fout[r * fb:(r + 1) * fb], prec, parity=m.ODD)
        want = oracle.dslash(s * parity_mask(dims, 0), U, dims, dagger=True, out_parity=1, tbc_anti=True)
        assert rel_err(got, want) <= TOL[prec], (prec, r)


@pytest.mark.parametrize("solver", [0, 1])
@pytest.mark.parametrize("prec", [1, 2, 3])
def test_mixed_solve(solver, prec):
    dims = (8, 8, 8, 16)
    m, wd, U = load(dims, True, seed=1000)
    b = li.gaussian_spinor(dims, 2000)
    x = np.zeros_like(b)
    r = wd.solve(x, b, 0.12, tol=1e-12, solver=solver, inner_precision=prec)
    rel = oracle.true_residual(x, b, U, dims, 0.12)
    assert r.status == 0 and rel <= 1e-12, (r, rel)


def test_singular_links_refused():
    """Unit links sit at |a1| = 1: the 8-number copy cannot hold them."""
    import paper_0911_3191_gb300 as m
    dims = (4, 4, 4, 8)
    wd = m.WilsonDirac(dims)
    wd.load_gauge(li.unit_gauge(dims), recon8=True)
    fin = wd.new_field(m.F32)
    fin.zero_()
    fout = wd.new_field(m.F32)
    with pytest.raises(m.WDError) as e:
        wd.dslash(fout, fin, 0, False, m.F32)
    assert e.value.status == 1
    # FP64 keeps its 12/18 reals and works
    f64 = wd.new_field(m.F64)
    f64.zero_()
    wd.dslash(wd.new_field(m.F64), f64, 0, False, m.F64)
