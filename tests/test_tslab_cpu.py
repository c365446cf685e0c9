"""The T-slab domain decomposition (paper_0911_3191_gb300/tslab.py) on CPU
ranks: gloo processes on 127.0.0.1, each holding one slab of the lattice,
exchange projected half-spinor faces and link slices, apply the FP64 oracle's
dslash to their extended slab and return the interior; the assembled result
equals the oracle's dslash of the whole lattice (periodic and antiperiodic
time, D and D^dag, both output parities).  Nothing here touches a GPU."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

DIMS = (4, 4, 2, 12)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import torch.distributed as dist
    if world > 1:
        dist.init_process_group("gloo", rank=rank, world_size=world)
    import lattice_inputs as li
    import oracle
    from paper_0911_3191_gb300 import tslab
    X, Y, Z, T = DIMS
    ss = X * Y * Z
    U = li.gauge(DIMS, 0.7, 1400)           # every rank generates the same field ...
    psi = li.gaussian_spinor(DIMS, 3800)
    t0, nt = tslab.slab_range(T, world, rank)
    U_slab = U[t0 * ss:(t0 + nt) * ss]      # ... and keeps only its slab
    psi_slab = psi[t0 * ss:(t0 + nt) * ss]
    res = {}
    U_lo = tslab.link_halo(U_slab, ss, rank, world)
    ext_dims = (X, Y, Z, nt + 2)
    U_ext = np.concatenate([U_lo, U_slab, np.zeros_like(U_slab[:ss])])  # the upper halo's links are not used
    for anti in (False, True):
        for dagger in (False, True):
            lo, hi = tslab.spinor_halos(psi_slab, ss, rank, world, dagger=dagger, antiperiodic=anti)
            psi_ext = np.concatenate([lo, psi_slab, hi])
            for parity in (0, 1):
                d = oracle.dslash(psi_ext, U_ext, ext_dims, dagger=dagger,
                                  out_parity=tslab.extended_parity(parity, t0))
                res[(anti, dagger, parity)] = d[ss:(nt + 1) * ss]
    out[rank] = res
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [1, 2, 3])
def test_slabs_reproduce_the_global_dslash(world):
    import lattice_inputs as li
    import oracle
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    if world == 1:
        _rank(0, 1, port, out)
    else:
        procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(180)
            assert p.exitcode == 0
    U = li.gauge(DIMS, 0.7, 1400)
    psi = li.gaussian_spinor(DIMS, 3800)
    for anti in (False, True):
        for dagger in (False, True):
            for parity in (0, 1):
                got = np.concatenate([out[r][(anti, dagger, parity)] for r in range(world)])
                want = oracle.dslash(psi, U, DIMS, dagger=dagger, out_parity=parity, tbc_anti=anti)
                assert np.linalg.norm(got - want) <= 1e-13 * np.linalg.norm(want), (world, anti, dagger, parity)


def test_faces_are_rank_two():
    """The exchanged face has 12 independent reals per site: P_{+-} has rank 2."""
    from paper_0911_3191_gb300 import tslab
    for s in (+1, -1):
        P = tslab.face_projector(s)
        np.testing.assert_allclose(P @ P, P, atol=1e-15)
        assert np.linalg.matrix_rank(P) == 2


def test_slab_ranges():
    from paper_0911_3191_gb300 import tslab
    assert [tslab.slab_range(12, 3, r) for r in range(3)] == [(0, 4), (4, 4), (8, 4)]
    with pytest.raises(ValueError):
        tslab.slab_range(12, 4, 0)  # slabs of 3 slices: odd


def _exchange_rank(rank, world, port, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import torch.distributed as dist
    if world > 1:
        dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_0911_3191_gb300 import tslab
    # distinct contents per rank and per face
    send_lo = torch.full((5,), 100.0 * rank + 1.0, dtype=torch.float64)
    send_hi = torch.full((5,), 100.0 * rank + 2.0, dtype=torch.float64)
    recv_lo, recv_hi = torch.zeros(5, dtype=torch.float64), torch.zeros(5, dtype=torch.float64)
    tslab.exchange_faces(send_lo, send_hi, recv_lo, recv_hi, rank, world)
    link_send = torch.full((3,), 100.0 * rank + 7.0, dtype=torch.float64)
    link_recv = torch.zeros(3, dtype=torch.float64)
    tslab.send_up(link_send, link_recv, rank, world)
    out[rank] = (recv_lo[0].item(), recv_hi[0].item(), link_recv[0].item())
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [1, 2, 3, 4])
def test_face_exchange_reaches_the_right_neighbours(world):
    """The exchange the GPU slab path uses (exchange_faces, send_up), on gloo
    ranks: each rank's lower halo is its lower neighbour's last-slice face,
    its upper halo the upper neighbour's first-slice face, its link halo the
    lower neighbour's link face (periodic in the rank index; with two ranks
    both neighbours are the same rank)."""
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    if world == 1:
        _exchange_rank(0, 1, port, out)
    else:
        procs = [ctx.Process(target=_exchange_rank, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
    for r in range(world):
        below, above = (r - 1) % world, (r + 1) % world
        assert out[r] == (100.0 * below + 2.0, 100.0 * above + 1.0, 100.0 * below + 7.0), (world, r, out[r])
