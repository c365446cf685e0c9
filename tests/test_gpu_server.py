"""Continuous-batching server (wd_server_*): requests of several lattice
volumes, kappas and tolerances, admitted as slots and memory free up, run
concurrently; every result is checked by the FP64 CPU oracle and must equal
the same solve done alone, within the solver tolerance: with both solutions
at |b - M x| <= tol |b|, the oracle's M applied to their difference is at
most 2 tol |b|."""
import numpy as np
import pytest

import lattice_inputs as li
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fields():
    a = (8, 8, 8, 16)
    b = (4, 6, 8, 10)
    return {a: li.gauge(a, 0.5, 1020), b: li.gauge(b, 0.5, 1021)}


def _drain(srv, ids, max_steps=100000):
    done = {}
    for _ in range(max_steps):
        active, queued = srv.step()
        for rid in list(ids):
            f, res, x = srv.poll(rid)
            if f:
                done[rid] = (res, x)
                ids.remove(rid)
        if not ids:
            return done
    raise AssertionError("requests did not finish")


def test_mixed_requests_match_solo_solves(fields):
    import paper_0911_3191_gb300 as m
    srv = m.Server(max_slots=4, iters_per_step=5, inner_precision=m.Q16)
    gids = {dims: srv.add_gauge(dims, U) for dims, U in fields.items()}
    rng = np.random.default_rng(7)
    reqs = []
    for k in range(9):
        dims = list(fields)[k % 2]
        b = li.gaussian_spinor(dims, 2200 + k)
        kappa = float(rng.uniform(0.115, 0.124))
        tol = [1e-8, 1e-10, 1e-12][k % 3]
        rid = srv.submit(gids[dims], b, kappa, tol)
        reqs.append((rid, dims, b, kappa, tol))
    # more arrivals while the first ones are running
    srv.step()
    for k in range(9, 13):
        dims = list(fields)[k % 2]
        b = li.gaussian_spinor(dims, 2200 + k)
        rid = srv.submit(gids[dims], b, 0.12, 1e-12)
        reqs.append((rid, dims, b, 0.12, 1e-12))
    done = _drain(srv, [r[0] for r in reqs])
    for rid, dims, b, kappa, tol in reqs:
        res, x = done[rid]
        rel = oracle.true_residual(x, b, fields[dims], dims, kappa)
        assert res.status == 0 and rel <= tol, (rid, res, rel)
        solo = m.WilsonDirac(dims)
        solo.load_gauge(fields[dims])
        x1 = np.zeros_like(b)
        r1 = solo.solve(x1, b, kappa, tol=tol, inner_precision=m.Q16)
        assert r1.status == 0
        # the same result alone and in the mix, within the requested tolerance:
        # both meet |b - M x| <= tol |b|, so by the triangle inequality their
        # difference satisfies |M (x - x1)| <= 2 tol |b| (oracle operator)
        assert oracle.true_residual(x1, b, fields[dims], dims, kappa) <= tol
        dM = oracle.apply_M(x - x1, fields[dims], dims, kappa)
        assert np.linalg.norm(dM) <= 2 * tol * np.linalg.norm(b), (rid, np.linalg.norm(dM) / np.linalg.norm(b))
        solo.close()
    srv.close()


def test_budget_admits_as_memory_frees(fields):
    """A budget that holds the gauge fields and one solver slot: requests
    queue and are admitted one at a time, all finish."""
    import paper_0911_3191_gb300 as m
    dims = (8, 8, 8, 16)
    probe = m.Server(max_slots=1, inner_precision=m.F32)
    gid = probe.add_gauge(dims, fields[dims])
    fixed = probe.memory_in_use()
    probe.close()
    vh = li.volume(dims) // 2
    # one slot: 5 FP64 fields (source, Schur source, solution, residual work)
    # + 7 FP32 Krylov fields + control (~80 KB); two slots do not fit
    slot = 5 * 192 * vh + 7 * 96 * vh + 256 * 1024
    srv = m.Server(budget_bytes=fixed + slot, max_slots=4, iters_per_step=10, inner_precision=m.F32)
    gid = srv.add_gauge(dims, fields[dims])
    ids = []
    bs = {}
    for k in range(3):
        b = li.gaussian_spinor(dims, 2300 + k)
        rid = srv.submit(gid, b, 0.12, 1e-10)
        ids.append(rid)
        bs[rid] = b
    active, queued = srv.step()
    assert active == 1 and queued == 2
    assert srv.memory_in_use() <= fixed + slot
    done = _drain(srv, list(ids))
    for rid in ids:
        res, x = done[rid]
        assert res.status == 0
        assert oracle.true_residual(x, bs[rid], fields[dims], dims, 0.12) <= 1e-10
    srv.close()


def test_budget_too_small_is_refused(fields):
    import paper_0911_3191_gb300 as m
    dims = (8, 8, 8, 16)
    srv = m.Server(budget_bytes=1024, max_slots=2)
    with pytest.raises(m.WDError) as e:
        srv.add_gauge(dims, fields[dims])
    assert e.value.status == 8  # WD_ERR_BUDGET
    srv.close()


def test_pool_release_and_reallocation(fields):
    """A pool that drains releases its slot memory and allocates it again for
    the next request, while another pool keeps the device busy: every result
    still matches the oracle (the re-allocated control blocks are initialised
    in stream order)."""
    import paper_0911_3191_gb300 as m
    big, small = (8, 8, 8, 16), (4, 6, 8, 10)
    srv = m.Server(max_slots=2, iters_per_step=3, inner_precision=m.Q16)
    g_big, g_small = srv.add_gauge(big, fields[big]), srv.add_gauge(small, fields[small])
    busy = [srv.submit(g_big, li.gaussian_spinor(big, 2600 + k), 0.124, 1e-12) for k in range(6)]
    checks = []
    for k in range(8):
        b = li.gaussian_spinor(small, 2700 + k)
        rid = srv.submit(g_small, b, 0.12, 1e-10)
        res = _drain(srv, [rid])[rid]
        checks.append((b, res))
    _drain(srv, list(busy))
    for b, (res, x) in checks:
        rel = oracle.true_residual(x, b, fields[small], small, 0.12)
        assert res.status == 0 and rel <= 1e-10 and res.iters > 2, (res, rel)
    assert srv.stats()["retired"] == 14
    srv.close()


@pytest.mark.parametrize("rhs_tile", [-1, 1, 2, 4])
def test_rhs_tile_shapes(fields, rhs_tile):
    """Every inner multi-RHS dslash shape (one system per block row, or 1, 2,
    4 systems per link tile) gives oracle-correct solves, with more requests
    than slots and staggered tolerances (systems finish at different steps)."""
    import paper_0911_3191_gb300 as m
    dims = (8, 8, 8, 16)
    srv = m.Server(max_slots=3, iters_per_step=4, inner_precision=m.Q16, rhs_tile=rhs_tile, temporal_gauge=True)
    gid = srv.add_gauge(dims, fields[dims])
    reqs = []
    for k in range(5):
        b = li.gaussian_spinor(dims, 2800 + k)
        kappa, tol = 0.116 + 0.002 * k, [1e-8, 1e-12][k % 2]
        reqs.append((srv.submit(gid, b, kappa, tol), b, kappa, tol))
    done = _drain(srv, [r[0] for r in reqs])
    for rid, b, kappa, tol in reqs:
        res, x = done[rid]
        rel = oracle.true_residual(x, b, fields[dims], dims, kappa)
        assert res.status == 0 and rel <= tol, (rhs_tile, res, rel)
    srv.close()


def test_rhs_tile_refused():
    import paper_0911_3191_gb300 as m
    with pytest.raises(m.WDError):
        m.Server(rhs_tile=3)


def test_step_trace_and_prefetched_sources(fields, tmp_path, monkeypatch):
    """With WD_SERVER_TRACE set, the server writes one CSV row per step on
    destroy; with one slot and a queue, every source after the first is
    uploaded ahead (prefetch buffer) and every result still reaches its
    tolerance (checked by the oracle)."""
    import csv
    import paper_0911_3191_gb300 as m
    trace = tmp_path / "trace.csv"
    monkeypatch.setenv("WD_SERVER_TRACE", str(trace))
    dims = (8, 8, 8, 16)
    U = fields[dims]
    srv = m.Server(max_slots=1, iters_per_step=4, inner_precision=m.Q16)
    gid = srv.add_gauge(dims, U)
    bs = [li.gaussian_spinor(dims, 2600 + k) for k in range(4)]
    ids = [srv.submit(gid, b, 0.12, 1e-10) for b in bs]
    order = list(ids)
    done = _drain(srv, ids)
    steps = srv.stats()["steps"]
    srv.close()
    for rid, b in zip(order, bs):
        res, x = done[rid]
        assert res.status == 0 and oracle.true_residual(x, b, U, dims, 0.12) <= 1e-10
    lines = trace.read_text().splitlines()
    assert lines[0].startswith("# host buffers page-locked")
    rows = list(csv.DictReader(lines[1:]))
    assert len(rows) == steps
    assert sum(int(r["admitted"]) for r in rows) == 4
    assert all(r["dims"] == "8x8x8x16" and int(r["capacity"]) == 1 for r in rows)
    assert all(float(r["t_end_s"]) >= float(r["t_launch_s"]) > 0.0 for r in rows)
