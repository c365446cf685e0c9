"""Multi-right-hand-side dslash and batched solves (many sources and masses on
one gauge field; arXiv:0911.3191 Sec. 3 and 5), through the C ABI, checked by
the FP64 CPU oracle and against the single-right-hand-side path."""
import numpy as np
import pytest

import lattice_inputs as li
import oracle
from tests.wd_testutil import TOL, parity_mask, rel_err

pytestmark = pytest.mark.gpu

PRECS = [0, 1, 2, 3, 4]


@pytest.fixture(scope="module")
def lat():
    import paper_0911_3191_gb300 as m
    dims = (8, 6, 4, 16)
    U = li.gauge(dims, 0.5, 1010)
    wd = m.WilsonDirac(dims, t_antiperiodic=True)
    wd.load_gauge(U)
    return m, wd, dims, U


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("nrhs", [1, 5, 12])
@pytest.mark.parametrize("dagger", [False, True])
def test_dslash_batch_matches_oracle_and_single(lat, prec, nrhs, dagger):
    m, wd, dims, U = lat
    fb = wd.field_bytes(prec)
    srcs = [li.gaussian_spinor(dims, 5000 + r) for r in range(nrhs)]
    fin = wd.new_field(prec, nrhs)
    for r, s in enumerate(srcs):
        wd.field_import(fin[r * fb:(r + 1) * fb], s, m.EVEN, prec)
    fout = wd.new_field(prec, nrhs)
    wd.dslash_batch(fout, fin, nrhs, m.ODD, dagger, prec)
    single = wd.new_field(prec)
    for r, s in enumerate(srcs):
        got = wd.download(fout[r * fb:(r + 1) * fb], prec, parity=m.ODD)
        want = oracle.dslash(s * parity_mask(dims, 0), U, dims, dagger=dagger, out_parity=1, tbc_anti=True)
        assert rel_err(got, want) <= TOL[prec], (prec, r)
        wd.dslash(single, fin[r * fb:(r + 1) * fb], m.ODD, dagger, prec)
        one = wd.download(single, prec, parity=m.ODD)
        assert rel_err(got, one) <= max(TOL[prec], 1e-15) * (1 if prec <= 1 else 0.2)


@pytest.fixture(scope="module")
def batch_problem():
    import paper_0911_3191_gb300 as m
    dims = (8, 8, 8, 16)
    U = li.gauge(dims, 0.5, 1011)
    wd = m.WilsonDirac(dims)
    wd.load_gauge(U)
    # 3 point sources (spin-colour) and a Gaussian source, at two masses
    srcs = [li.point_source(dims, (0, 0, 0, 0), s, c) for s, c in ((0, 0), (1, 2), (3, 1))]
    srcs.append(li.gaussian_spinor(dims, 2100))
    kappas = [0.118, 0.124]
    bs = [s for k in kappas for s in srcs]
    ks = [k for k in kappas for _ in srcs]
    return m, wd, dims, U, bs, ks


def _upload_batch(m, wd, bs):
    n = len(bs)
    full = 2 * wd.field_bytes(m.F64)
    fb = wd.new_field(m.F64, 2 * n)
    for r, b in enumerate(bs):
        fb[r * full:(r + 1) * full].copy_(wd.upload(b, m.F64))
    return fb


@pytest.mark.parametrize("prec", PRECS)
def test_batched_solve_every_system_converges(batch_problem, prec):
    m, wd, dims, U, bs, ks = batch_problem
    n = len(bs)
    fb = _upload_batch(m, wd, bs)
    fx = wd.new_field(m.F64, 2 * n)
    infos = wd.solve_batch_device(fx, fb, ks, tol=1e-12, inner_precision=prec)
    full = 2 * wd.field_bytes(m.F64)
    for r in range(n):
        x = wd.download(fx[r * full:(r + 1) * full], m.F64)
        rel = oracle.true_residual(x, bs[r], U, dims, ks[r])
        assert infos[r].status == 0 and rel <= 1e-12, (r, infos[r], rel)
        assert abs(infos[r].true_rel_residual - rel) <= 0.05 * rel + 1e-16
        if prec != 0:
            assert infos[r].reliable_updates >= 2


def test_each_system_alone_equals_in_batch(batch_problem):
    """Batch invariance: a system gives the same answer alone and in the mix
    (to the solver tolerance; the kernels differ, so not bit for bit)."""
    m, wd, dims, U, bs, ks = batch_problem
    n = len(bs)
    xs = [np.zeros_like(b) for b in bs]
    infos = wd.solve_batch(xs, bs, ks, tol=1e-12, inner_precision=m.Q16)
    for r in (0, 3, 5, 7):
        x1 = np.zeros_like(bs[r])
        one = wd.solve(x1, bs[r], ks[r], tol=1e-12, inner_precision=m.Q16)
        assert one.status == 0 and infos[r].status == 0
        assert np.linalg.norm(xs[r] - x1) / np.linalg.norm(x1) < 1e-9
        # and the batch of one equals the batch of n for that system
    solo = wd.solve_batch([np.zeros_like(bs[5])], [bs[5]], [ks[5]], tol=1e-12, inner_precision=m.Q16)
    assert solo[0].status == 0


def test_batch_graph_equals_host_loop(batch_problem):
    m, wd, dims, U, bs, ks = batch_problem
    n = len(bs)
    fb = _upload_batch(m, wd, bs)
    outs = []
    for g in (True, False):
        fx = wd.new_field(m.F64, 2 * n)
        infos = wd.solve_batch_device(fx, fb, ks, tol=1e-11, inner_precision=m.B16N, use_graph=g)
        outs.append((fx.cpu().numpy(), [(i.iters, i.reliable_updates) for i in infos]))
    assert outs[0][1] == outs[1][1]
    np.testing.assert_array_equal(outs[0][0], outs[1][0])


def test_batch_with_zero_source(batch_problem):
    m, wd, dims, U, bs, ks = batch_problem
    b2 = [bs[0], np.zeros_like(bs[0]), bs[3]]
    xs = [np.ones_like(b) for b in b2]
    infos = wd.solve_batch(xs, b2, [0.12, 0.12, 0.12], tol=1e-10, inner_precision=m.F32)
    assert all(i.status == 0 for i in infos)
    assert np.all(xs[1] == 0)
    assert oracle.true_residual(xs[2], b2[2], U, dims, 0.12) <= 1e-10


@pytest.mark.parametrize("prec", [0, 2, 4])
def test_per_system_shape(tmp_path, monkeypatch, prec):
    """The batched dslash and solver with the inner dslash forced to one system
    per block row (a tuning-cache entry with tile 0) agree with the oracle."""
    import paper_0911_3191_gb300 as m
    dims = (8, 6, 4, 16)
    U = li.gauge(dims, 0.5, 1012)
    nrhs = 3
    cache = tmp_path / "tune.txt"
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    cache.write_text(f"{dims[0]}x{dims[1]}x{dims[2]}x{dims[3]} prec{prec} n{nrhs} sms{sms} links12 tfix1|0 8\n")
    monkeypatch.setenv("WD_TUNE_CACHE", str(cache))
    wd = m.WilsonDirac(dims, t_antiperiodic=True)
    wd.load_gauge(U, temporal_gauge=True)
    srcs = [li.gaussian_spinor(dims, 5100 + r) for r in range(nrhs)]
    kappas = [0.118, 0.121, 0.124]
    xs = [np.zeros_like(b) for b in srcs]
    infos = wd.solve_batch(xs, srcs, kappas, tol=1e-10, inner_precision=prec)
    for x, b, k, info in zip(xs, srcs, kappas, infos):
        rel = oracle.true_residual(x, b, U, dims, k, tbc_anti=True)
        assert info.status == 0 and rel <= 1e-10, (prec, k, info, rel)
    # the tuned shape (tile 0) now also drives wd_dslash_batch for n = 3
    fb = wd.field_bytes(prec)
    fin = wd.new_field(prec, nrhs)
    for r, s in enumerate(srcs):
        wd.field_import(fin[r * fb:(r + 1) * fb], s, m.EVEN, prec)
    fout = wd.new_field(prec, nrhs)
    wd.dslash_batch(fout, fin, nrhs, m.ODD, True, prec)
    for r, s in enumerate(srcs):
        got = wd.download(fout[r * fb:(r + 1) * fb], prec, parity=m.ODD)
        want = oracle.dslash(s * parity_mask(dims, 0), U, dims, dagger=True, out_parity=1, tbc_anti=True)
        assert rel_err(got, want) <= TOL[prec], (prec, r)
    # the pinned entry was used: the tuner appended no line of its own
    assert cache.read_text().count("\n") == 1 and "|0 8" in cache.read_text()


@pytest.mark.parametrize("prec", [1, 2, 3, 4])
@pytest.mark.parametrize("tr", [2, 4, 8])
def test_packed_pairs_shape(tmp_path, monkeypatch, prec, tr):
    """Two systems per thread in FP32x2 registers (a tuning-cache entry with
    the packed layout): the batched dslash for an odd number of systems (one
    system of the last pair rides along unwritten) agrees with the oracle and
    with the single-system kernel, and a batched solve reaches its tolerance
    for every system."""
    import torch

    import paper_0911_3191_gb300 as m
    dims = (8, 6, 4, 16)
    U = li.gauge(dims, 0.5, 1013)
    nrhs = 5
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    cache = tmp_path / "tune.txt"
    cache.write_text(f"{dims[0]}x{dims[1]}x{dims[2]}x{dims[3]} prec{prec} n{nrhs} sms{sms} links12 tfix0|{tr} 16 1\n")
    monkeypatch.setenv("WD_TUNE_CACHE", str(cache))
    wd = m.WilsonDirac(dims, t_antiperiodic=True)
    wd.load_gauge(U)
    srcs = [li.gaussian_spinor(dims, 5200 + r) for r in range(nrhs)]
    kappas = [0.118, 0.12, 0.121, 0.123, 0.124]
    xs = [np.zeros_like(b) for b in srcs]
    infos = wd.solve_batch(xs, srcs, kappas, tol=1e-10, inner_precision=prec)
    for x, b, k, info in zip(xs, srcs, kappas, infos):
        rel = oracle.true_residual(x, b, U, dims, k, tbc_anti=True)
        assert info.status == 0 and rel <= 1e-10, (prec, tr, k, info, rel)
    fb = wd.field_bytes(prec)
    fin = wd.new_field(prec, nrhs)
    for r, s in enumerate(srcs):
        wd.field_import(fin[r * fb:(r + 1) * fb], s, m.EVEN, prec)
    single = wd.new_field(prec)
    for dagger in (False, True):
        fout = wd.new_field(prec, nrhs)
        wd.dslash_batch(fout, fin, nrhs, m.ODD, dagger, prec)
        for r, s in enumerate(srcs):
            got = wd.download(fout[r * fb:(r + 1) * fb], prec, parity=m.ODD)
            want = oracle.dslash(s * parity_mask(dims, 0), U, dims, dagger=dagger, out_parity=1, tbc_anti=True)
            assert rel_err(got, want) <= TOL[prec], (prec, tr, r, dagger)
            wd.dslash(single, fin[r * fb:(r + 1) * fb], m.ODD, dagger, prec)
            assert rel_err(got, wd.download(single, prec, parity=m.ODD)) <= TOL[prec] * (1 if prec <= 1 else 0.2)
    assert cache.read_text().count("\n") == 1 and f"|{tr} 16 1" in cache.read_text()
    wd.close()
