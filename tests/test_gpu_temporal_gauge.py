"""Temporal gauge fixing inside the library (arXiv:0911.3191 Sec. 4.3):
wd_load_gauge_opt(.., temporal_gauge=1) transforms the links so that U_4 = 1
off the last time slice and keeps device fields in the transformed frame.

Pins: the device field after import equals G (S psi) with G(x, t) =
U_4(x, 0) ... U_4(x, t-1) built here with numpy from its definition; every
result seen through the host layout (dslash, M, M_hat, solves, batches,
serving) equals the FP64 oracle on the untransformed links."""
import numpy as np
import pytest

import lattice_inputs as li
import oracle
from tests.wd_testutil import TOL, parity_mask, parity_sites, rel_err, to_internal_basis

pytestmark = pytest.mark.gpu

PRECS = [0, 1, 2, 3, 4]
DIMS = [(4, 6, 8, 10), (8, 6, 4, 16)]


def fixed(dims, anti=False, recon=12, seed=1200, eps=0.5):
    import paper_0911_3191_gb300 as m
    U = li.gauge(dims, eps, seed)
    wd = m.WilsonDirac(dims, t_antiperiodic=anti)
    wd.load_gauge(U, recon=recon, temporal_gauge=True)
    return m, wd, U


def temporal_transform(U, dims):
    """G(x, t) = U_4(x, 0) U_4(x, 1) ... U_4(x, t-1), G(x, 0) = 1 (numpy)."""
    X, Y, Z, T = dims
    ns = X * Y * Z
    U4 = U.reshape(T, ns, 4, 3, 3)[:, :, 3]
    G = np.empty((T, ns, 3, 3), dtype=np.complex128)
    G[0] = np.eye(3)
    for t in range(1, T):
        G[t] = G[t - 1] @ U4[t - 1]
    return G.reshape(T * ns, 3, 3)


@pytest.mark.parametrize("dims", DIMS)
def test_import_applies_G(dims):
    """F64 device field = G S psi on every site (the transformation itself)."""
    m, wd, U = fixed(dims)
    psi = li.gaussian_spinor(dims, 3600)
    G = temporal_transform(U, dims)
    want = np.einsum("sij,saj->sai", G, to_internal_basis(psi))
    for parity in (0, 1):
        f = wd.upload(psi, m.F64, parity=parity)
        vh = li.volume(dims) // 2
        st = (vh + 31) // 32 * 32
        raw = f.cpu().numpy().view(np.complex128).reshape(12, st)[:, :vh].T.reshape(vh, 4, 3)
        sites = parity_sites(dims, parity)
        assert rel_err(raw, want[sites]) < 1e-14
        # and export undoes it
        back = wd.download(f, m.F64, parity=parity)[sites]
        assert rel_err(back, psi[sites]) < 1e-14


def test_unit_temporal_links_and_polyakov_slice():
    """The transformed temporal links: 1 off t = T-1; on t = T-1 the product
    of U_4 around the time direction (the gauge-invariant Polyakov line), seen
    through the operator: a point source at t = T-1 hopping forward."""
    dims = (4, 4, 4, 8)
    m, wd, U = fixed(dims, recon=18)
    for t in (2, dims[3] - 1):
        src = li.point_source(dims, site=(1, 2, 3, t), spin=0, colour=1)
        out_parity = 1 - (1 + 2 + 3 + t) % 2
        fin = wd.upload(src, m.F64, parity=1 - out_parity)
        fout = wd.new_field(m.F64)
        wd.dslash(fout, fin, out_parity, False, m.F64)
        got = wd.download(fout, m.F64, parity=out_parity)
        want = oracle.dslash(src, U, dims, out_parity=out_parity)
        assert rel_err(got, want) < 1e-13


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("dims", DIMS)
@pytest.mark.parametrize("dagger", [False, True])
@pytest.mark.parametrize("anti", [False, True])
def test_dslash_matches_oracle(prec, dims, dagger, anti):
    m, wd, U = fixed(dims, anti=anti, seed=1210 + prec)
    psi = li.gaussian_spinor(dims, 3610 + prec)
    for out_parity in (0, 1):
        fin = wd.upload(psi, prec, parity=1 - out_parity)
        fout = wd.new_field(prec)
        wd.dslash(fout, fin, out_parity, dagger, prec)
        got = wd.download(fout, prec, parity=out_parity)
        want = oracle.dslash(psi * parity_mask(dims, 1 - out_parity), U, dims, dagger=dagger,
                             out_parity=out_parity, tbc_anti=anti)
        assert rel_err(got, want) <= TOL[prec], (prec, dims, dagger, anti, out_parity)


@pytest.mark.parametrize("prec", PRECS)
def test_apply_M_and_Mhat(prec):
    dims = (8, 6, 4, 16)
    m, wd, U = fixed(dims, anti=True, recon=18)
    psi = li.gaussian_spinor(dims, 3620)
    kappa = 0.124
    fin = wd.upload(psi, prec)
    fout = wd.new_field(prec, 2)
    wd.apply_M(fout, fin, kappa, m.M_FULL, False, prec)
    assert rel_err(wd.download(fout, prec), oracle.apply_M(psi, U, dims, kappa, tbc_anti=True)) <= TOL[prec]
    fe = wd.upload(psi, prec, parity=0)
    fo = wd.new_field(prec)
    wd.apply_M(fo, fe, kappa, m.M_SCHUR_EVEN, True, prec)
    want = oracle.apply_Mhat(psi * parity_mask(dims, 0), U, dims, kappa, dagger=True, tbc_anti=True)
    assert rel_err(wd.download(fo, prec, parity=0), want) <= TOL[prec]


@pytest.mark.parametrize("solver", [0, 1])
@pytest.mark.parametrize("prec", [0, 1, 2])
def test_solve_true_residual(solver, prec):
    dims = (8, 8, 8, 16)
    m, wd, U = fixed(dims, recon=18, seed=1000)
    b = li.gaussian_spinor(dims, 2000)
    kappa = 0.12
    x = np.zeros_like(b)
    r = wd.solve(x, b, kappa, tol=1e-12, solver=solver, inner_precision=prec)
    rel = oracle.true_residual(x, b, U, dims, kappa)
    assert r.status == 0 and rel <= 1e-12, (r, rel)
    assert abs(r.true_rel_residual - rel) <= 0.05 * rel + 1e-15
    x_ref, st, _, _ = oracle.solve(b, U, dims, kappa, tol=1e-12)
    assert np.linalg.norm(x - x_ref) / np.linalg.norm(x_ref) < 1e-9


@pytest.mark.parametrize("prec", [0, 2])
@pytest.mark.parametrize("nrhs", [1, 5])
def test_dslash_batch(prec, nrhs):
    dims = (8, 6, 4, 16)
    m, wd, U = fixed(dims, anti=True)
    fb = wd.field_bytes(prec)
    srcs = [li.gaussian_spinor(dims, 3630 + r) for r in range(nrhs)]
    fin = wd.new_field(prec, nrhs)
    for r, s in enumerate(srcs):
        wd.field_import(fin[r * fb:(r + 1) * fb], s, m.EVEN, prec)
    fout = wd.new_field(prec, nrhs)
    wd.dslash_batch(fout, fin, nrhs, m.ODD, False, prec)
    for r, s in enumerate(srcs):
        got = wd.download(fout[r * fb:(r + 1) * fb], prec, parity=m.ODD)
        want = oracle.dslash(s * parity_mask(dims, 0), U, dims, out_parity=1, tbc_anti=True)
        assert rel_err(got, want) <= TOL[prec], (prec, r)


def test_batched_solve():
    dims = (8, 8, 8, 16)
    m, wd, U = fixed(dims, recon=18, seed=1011)
    bs = [li.point_source(dims, (0, 0, 0, 0), s, c) for s, c in ((0, 0), (2, 1))] + [li.gaussian_spinor(dims, 2100)]
    ks = [0.118, 0.124, 0.121]
    xs = [np.zeros_like(b) for b in bs]
    infos = wd.solve_batch(xs, bs, ks, tol=1e-12, inner_precision=m.Q16)
    for x, b, k, info in zip(xs, bs, ks, infos):
        rel = oracle.true_residual(x, b, U, dims, k)
        assert info.status == 0 and rel <= 1e-12, (k, info, rel)


def test_server_requests():
    import paper_0911_3191_gb300 as m
    dims = (8, 8, 8, 16)
    U = li.gauge(dims, 0.3, 1020)
    srv = m.Server(max_slots=4, iters_per_step=4, inner_precision=m.Q16, temporal_gauge=True)
    gid = srv.add_gauge(dims, U, recon=18)
    reqs = []
    for i, k in enumerate((0.12, 0.122, 0.124)):
        b = li.gaussian_spinor(dims, 2200 + i)
        reqs.append((srv.submit(gid, b, k, 1e-10), b, k))
    pending = [r[0] for r in reqs]
    done = {}
    for _ in range(100000):
        srv.step()
        for rid in list(pending):
            f, res, x = srv.poll(rid)
            if f:
                done[rid] = (res, x)
                pending.remove(rid)
        if not pending:
            break
    assert not pending
    for rid, b, k in reqs:
        res, x = done[rid]
        assert res.status == 0
        assert oracle.true_residual(x, b, U, dims, k) <= 1e-10
    srv.close()
