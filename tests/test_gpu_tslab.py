"""GPU side of the T-slab decomposition (the multi-GPU layout the paper names
as its next step, Sec. 6), through the C ABI, against the FP64 CPU oracle.

* One rank (world = 1): SlabDslash on the whole lattice, with the face pack
  kernel, the self-exchange of the projected faces on a second stream, the
  interior launch overlapping it and the boundary-slice launch reading the
  halo buffers, equals the oracle's dslash (periodic and antiperiodic time,
  D and D^dag, both output parities, every precision) at the dslash bars.
* Several ranks on one GPU: each rank's slab in its own context, the faces
  moved between the ranks' buffers by device copies in between launches
  (no kernel waits on another): the assembled output equals the oracle's
  dslash of the whole lattice.
* The interior and boundary launches together write exactly what one launch
  over all slab sites writes, and agree with the whole-lattice dslash kernel
  to rounding."""
import numpy as np
import pytest

import lattice_inputs as li
import oracle
from tests.wd_testutil import TOL, parity_mask, rel_err

pytestmark = pytest.mark.gpu

PRECS = [0, 1, 2, 3, 4]


@pytest.fixture(scope="module")
def wdp():
    import paper_0911_3191_gb300 as m
    m.load_library()
    return m


_cache = {}


def whole(dims, seed=1500):
    """One context holding the whole lattice as one slab (its own links)."""
    key = (dims, seed)
    if key not in _cache:
        import paper_0911_3191_gb300 as m
        U = li.gauge(dims, 0.5, seed)
        wd = m.WilsonDirac(dims)
        wd.load_gauge(U)
        _cache[key] = (wd, U)
    return _cache[key]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("dims", [(8, 6, 4, 12), (4, 6, 8, 10), (6, 4, 2, 2)])
@pytest.mark.parametrize("dagger", [False, True])
@pytest.mark.parametrize("anti", [False, True])
def test_one_rank_slab_matches_oracle(wdp, prec, dims, dagger, anti):
    from paper_0911_3191_gb300.tslab import SlabDslash
    wd, U = whole(dims)
    sd = SlabDslash(wd, 0, 1, t_antiperiodic=anti)
    psi = li.gaussian_spinor(dims, 2500 + prec)
    for p in (0, 1):
        fin = wd.upload(psi, prec, parity=1 - p)
        fout = wd.new_field(prec)
        sd.apply(fout, fin, p, dagger, prec)
        got = wd.download(fout, prec, parity=p)
        want = oracle.dslash(psi * parity_mask(dims, 1 - p), U, dims, dagger=dagger, out_parity=p, tbc_anti=anti)
        assert rel_err(got, want) <= TOL[prec], (prec, dims, dagger, anti, p, rel_err(got, want))


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("anti", [False, True])
def test_ranks_on_one_gpu_reproduce_the_global_dslash(wdp, prec, world, anti):
    """world slabs of (8, 6, 4, 4): T = 4 world.  Faces move between the
    ranks' device buffers by copies between launches."""
    import torch

    from paper_0911_3191_gb300 import tslab
    X, Y, Z, nt = 8, 6, 4, 4
    T = nt * world
    dims = (X, Y, Z, T)
    ss = X * Y * Z
    U = li.gauge(dims, 0.5, 1600 + world)
    psi = li.gaussian_spinor(dims, 2600 + prec)
    ranks = []
    for r in range(world):
        t0, n = tslab.slab_range(T, world, r)
        wd = wdp.WilsonDirac((X, Y, Z, n))
        wd.load_gauge(np.ascontiguousarray(U[t0 * ss:(t0 + n) * ss]))
        ranks.append((wd, t0, n))
    for dagger in (False, True):
        for p in (0, 1):
            fins, faces, links = [], [], []
            for wd, t0, n in ranks:
                fin = wd.upload(np.ascontiguousarray(psi[t0 * ss:(t0 + n) * ss]), prec, parity=1 - p)
                nf = wd.slab_face_bytes(prec)
                lo = torch.empty(nf, dtype=torch.uint8, device="cuda")
                hi = torch.empty_like(lo)
                wd.slab_pack_faces(lo, hi, fin, dagger, prec)
                link = torch.empty(wd.slab_link_face_bytes(prec), dtype=torch.uint8, device="cuda")
                wd.slab_pack_link_face(link, prec)
                fins.append(fin)
                faces.append((lo, hi))
                links.append(link)
            torch.cuda.synchronize()
            got = np.zeros((li.volume(dims), 4, 3), dtype=np.complex128)
            for r, (wd, t0, n) in enumerate(ranks):
                below, above = (r - 1) % world, (r + 1) % world
                halo_lo = faces[below][1].clone()   # the lower neighbour's last slice
                halo_hi = faces[above][0].clone()   # the upper neighbour's first slice
                link_halo = links[below].clone()
                lo_sign, hi_sign = tslab.halo_signs(r, world, anti)
                fout = wd.new_field(prec)
                wd.dslash_slab(fout, fins[r], halo_lo, halo_hi, link_halo, lo_sign < 0, hi_sign < 0, p, dagger,
                               prec, 2)
                got[t0 * ss:(t0 + n) * ss] = wd.download(fout, prec, parity=p)
            want = oracle.dslash(psi * parity_mask(dims, 1 - p), U, dims, dagger=dagger, out_parity=p, tbc_anti=anti)
            assert rel_err(got, want) <= TOL[prec], (prec, world, anti, dagger, p, rel_err(got, want))
    for wd, _, _ in ranks:
        wd.close()


@pytest.mark.parametrize("prec", PRECS)
def test_interior_plus_boundary_equals_one_launch(wdp, prec):
    import torch

    from paper_0911_3191_gb300.tslab import SlabDslash
    dims = (8, 6, 4, 12)
    wd, U = whole(dims)
    sd = SlabDslash(wd, 0, 1, t_antiperiodic=True)
    psi = li.gaussian_spinor(dims, 2700 + prec)
    fin = wd.upload(psi, prec, parity=1)
    # the same fill everywhere, so padding compares equal and a site that no
    # launch wrote would show
    a, b = wd.new_field(prec), wd.new_field(prec)
    a.fill_(0x5A)
    b.fill_(0x5A)
    sd.apply(a, fin, 0, False, prec)            # region 0 then region 1
    lo, hi, halo_lo, halo_hi = sd.faces(prec)
    wd.dslash_slab(b, fin, halo_lo, halo_hi, sd.link_halo(prec), sd.flip_lo, sd.flip_hi, 0, False, prec, 2)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    # the whole-lattice kernel (antiperiodic context) computes the same hops
    # in the same order; the two kernels may contract multiply-adds
    # differently, so the comparison is to rounding: FP64 / FP32 to a few
    # ulp, 16-bit storage element by element to one unit in the last place
    # of the format at the site's norm (a rounding difference can move a
    # code by one), and such moves must stay rare
    import paper_0911_3191_gb300 as m
    wa = m.WilsonDirac(dims, t_antiperiodic=True)
    wa.load_gauge(U)
    fin2 = wa.upload(psi, prec, parity=1)
    c = wa.new_field(prec)
    wa.dslash(c, fin2, 0, False, prec)
    ev = li.parity(dims) == 0
    ga = wd.download(a, prec, parity=0)[ev].reshape(-1, 12)
    gc = wa.download(c, prec, parity=0)[ev].reshape(-1, 12)
    if prec <= 1:
        assert rel_err(ga, gc) <= (1e-14 if prec == 0 else 1e-6)
    else:
        ulp = {2: 1.0 / 32767, 3: 2.0 ** -10, 4: 2.0 ** -7}[prec]
        va, vc = ga.view(np.float64), gc.view(np.float64)
        norm = np.abs(vc).max(axis=1, keepdims=True)
        diff = np.abs(va - vc)
        assert np.all(diff <= 1.01 * ulp * norm)
        # a norm that differs in its last bit moves a whole site by ~1e-7
        # relative; moves of a code are the ones that must be rare
        assert np.count_nonzero(diff > 1e-5 * norm) <= 0.01 * diff.size
    wa.close()


def test_slab_refuses_the_temporal_gauge(wdp):
    import torch
    dims = (4, 4, 4, 6)
    wd = wdp.WilsonDirac(dims)
    wd.load_gauge(li.gauge(dims, 0.5, 1700), temporal_gauge=True)
    buf = torch.empty(wd.slab_face_bytes(2), dtype=torch.uint8, device="cuda")
    fin = wd.new_field(2)
    with pytest.raises(wdp.WDError):
        wd.slab_pack_faces(buf, buf.clone(), fin, False, 2)
    wd.close()
