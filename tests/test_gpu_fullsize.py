"""Parity at the full workload sizes, in the launch configuration the
benchmark times (arXiv:0911.3191 Sec. 4-5):

* the 24^3x64 and 64^3x128 dslash, every storage precision, compared with the
  FP64 oracle on sampled output sites (random ones plus every kind of
  boundary and corner site), which the oracle computes one by one;
* the 64^3x128 mixed CGNR solve (Q16 inner, FP64 reliable updates) to 1e-10,
  checked by one oracle application of M_kappa on the whole lattice;
* the 48 systems of the 32^3x64 batch (12 point sources x 4 kappa), each
  checked by the oracle's true residual.

Host memory: the 64^3x128 cases hold the FP64 links (19.3 GB) plus a few
6.4 GB fields; they are skipped on hosts with less than 96 GB available."""
import numpy as np
import pytest

import lattice_inputs as li
import oracle
from tests.wd_testutil import TOL, rel_err

pytestmark = pytest.mark.gpu

PRECS = [0, 1, 2, 3, 4]


def _mem_available_gb():
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) / 2**20
    except OSError:
        pass
    return 0.0


def sample_sites(dims, parity, n, seed):
    """n random sites of one parity plus all boundary/corner patterns."""
    X, Y, Z, T = dims
    rng = np.random.default_rng(seed)
    pts = [rng.integers(0, d, size=n) for d in dims]
    x, y, z, t = pts
    edge = []
    for cx in (0, X - 1):
        for cy in (0, Y - 1):
            for cz in (0, Z - 1):
                for ct in (0, T - 1):
                    edge.append((cx, cy, cz, ct))
                    edge.append((cx, cy // 2, cz // 2, ct))
                    edge.append((X // 2, cy, cz, T // 2))
    e = np.array(edge).T
    x, y, z, t = (np.concatenate([a, b]) for a, b in zip((x, y, z, t), e))
    # move each site onto the requested parity by stepping x by one
    wrong = (x + y + z + t) % 2 != parity
    x = np.where(wrong, (x + 1) % X, x)
    s = np.unique(li.lex_index(dims, x, y, z, t))
    assert np.all(li.parity(dims)[s] == parity)
    return s


def dslash_sampled(dims, seed_u, recon, cases):
    import paper_0911_3191_gb300 as m
    U = li.gauge(dims, 0.3, seed_u)
    wd = m.WilsonDirac(dims)
    wd.load_gauge(U, recon=recon)
    psi = li.gaussian_spinor(dims, 2100)
    try:
        for prec, out_parity, dagger in cases:
            sites = sample_sites(dims, out_parity, 2048, 7 + prec)
            fin = wd.upload(psi, prec, parity=1 - out_parity)
            fout = wd.new_field(prec)
            wd.dslash(fout, fin, out_parity, dagger, prec)
            del fin
            got = wd.download(fout, prec, parity=out_parity)[sites]
            del fout
            # D couples opposite parities only: the full psi gives D psi_{1-p} at sites of parity p
            want = oracle.dslash_sites(psi, U, dims, sites, dagger=dagger)
            err = rel_err(got, want)
            assert err <= TOL[prec], (dims, prec, out_parity, dagger, err)
    finally:
        wd.close()


def test_dslash_24x64_sampled():
    cases = [(p, op, dg) for p in PRECS for op in (0, 1) for dg in (False, True)]
    dslash_sampled((24, 24, 24, 64), 1001, 18, cases)
    dslash_sampled((24, 24, 24, 64), 1001, 12, [(p, 0, False) for p in PRECS])


@pytest.mark.skipif(_mem_available_gb() < 96, reason="needs ~96 GB of host memory")
def test_dslash_64x128_sampled():
    cases = [(p, 0, False) for p in PRECS] + [(0, 1, True), (2, 1, True)]
    dslash_sampled((64, 64, 64, 128), 1002, 18, cases)


@pytest.mark.skipif(_mem_available_gb() < 96, reason="needs ~96 GB of host memory")
def test_cgnr_q16_64x128_true_residual():
    """The large-lattice mixed solve: CGNR on M_hat^dag M_hat, Q16 inner, FP64
    reliable updates (delta 0.1), tol 1e-10 (relative to |b|)."""
    import paper_0911_3191_gb300 as m
    dims = (64, 64, 64, 128)
    kappa = 0.124
    U = li.gauge(dims, 0.3, 1002)
    b = li.gaussian_spinor(dims, 2002)
    wd = m.WilsonDirac(dims)
    try:
        wd.load_gauge(U, recon=18)
        x = np.zeros_like(b)
        r = wd.solve(x, b, kappa, tol=1e-10, delta=0.1, solver=m.CGNR, inner_precision=m.Q16)
    finally:
        wd.close()
    assert r.status == 0 and r.reliable_updates >= 2, r
    rel = oracle.true_residual(x, b, U, dims, kappa)
    assert rel <= 1e-10, (r, rel)
    assert abs(r.true_rel_residual - rel) <= 0.05 * rel


@pytest.mark.skipif(_mem_available_gb() < 64, reason="needs ~64 GB of host memory")
def test_batch_48_systems_32x64():
    """12 point sources (origin, every spin and colour) x kappa in {0.118,
    0.12, 0.122, 0.124}, Q16 inner BiCGstab with FP64 reliable updates to
    1e-12, all 48 in one batched solve; every system's true residual is
    recomputed by the oracle."""
    import paper_0911_3191_gb300 as m
    dims = (32, 32, 32, 64)
    kappas = [0.118, 0.12, 0.122, 0.124]
    U = li.gauge(dims, 0.3, 1003)
    wd = m.WilsonDirac(dims)
    try:
        wd.load_gauge(U, recon=18)
        bs, ks = [], []
        for k in kappas:
            for s in range(4):
                for c in range(3):
                    bs.append(li.point_source(dims, spin=s, colour=c))
                    ks.append(k)
        xs = [np.zeros_like(bs[0]) for _ in bs]
        infos = wd.solve_batch(xs, bs, ks, tol=1e-12, inner_precision=m.Q16)
    finally:
        wd.close()
    for i, (x, b, k, info) in enumerate(zip(xs, bs, ks, infos)):
        rel = oracle.true_residual(x, b, U, dims, k)
        assert info.status == 0 and rel <= 1e-12, (i, k, info, rel)
