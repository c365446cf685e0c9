"""GPU parity of the dslash, M and M_hat and of the storage codecs against
the FP64 CPU oracle, through the C ABI (arXiv:0911.3191 Sec. 3-4, App. A-B).

Bars: relative L2 error <= 1e-13 (FP64), 1e-6 (FP32), 5e-3 (16-bit storage)
against the oracle on unquantised FP64 inputs; bit-exact codes and norms for
the 16-bit codecs (Sec. 4.6)."""
import numpy as np
import pytest

import lattice_inputs as li
import oracle
from tests.wd_testutil import TOL, parity_mask, parity_sites, rel_err, split16, to_host_basis, to_internal_basis

pytestmark = pytest.mark.gpu

PRECS = [0, 1, 2, 3, 4]  # F64, F32, Q16, H16N, B16N
# several tiles plus ragged tails (Vh = 128, 960, 4096, 1536, 8)
DIMS = [(4, 4, 4, 4), (4, 6, 8, 10), (8, 8, 8, 16), (8, 6, 4, 16), (2, 2, 2, 4)]


@pytest.fixture(scope="module")
def wdp():
    import paper_0911_3191_gb300 as m
    m.load_library()
    return m


_cache = {}


def lattice(dims, eps=0.5, anti=False):
    key = (dims, eps, anti)
    if key not in _cache:
        import paper_0911_3191_gb300 as m
        U = li.gauge(dims, eps, 1000 + len(_cache))
        wd = m.WilsonDirac(dims, t_antiperiodic=anti)
        wd.load_gauge(U)
        _cache[key] = (wd, U)
    return _cache[key]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("dims", DIMS)
@pytest.mark.parametrize("dagger", [False, True])
@pytest.mark.parametrize("out_parity", [0, 1])
def test_dslash_matches_oracle(wdp, prec, dims, dagger, out_parity):
    anti = (dims[3] % 4 == 0) and out_parity == 1
    wd, U = lattice(dims, anti=anti)
    psi = li.gaussian_spinor(dims, 2000 + prec)
    src = psi * parity_mask(dims, 1 - out_parity)
    fin = wd.upload(psi, prec, parity=1 - out_parity)
    fout = wd.new_field(prec)
    wd.dslash(fout, fin, out_parity, dagger, prec)
    got = wd.download(fout, prec, parity=out_parity)
    want = oracle.dslash(src, U, dims, dagger=dagger, out_parity=out_parity, tbc_anti=anti)
    assert rel_err(got, want) <= TOL[prec], (prec, dims, dagger, out_parity, rel_err(got, want))


@pytest.mark.parametrize("prec", PRECS)
def test_dslash_xpay(wdp, prec):
    dims = (4, 6, 8, 10)
    wd, U = lattice(dims)
    psi = li.gaussian_spinor(dims, 3000)
    x = li.gaussian_spinor(dims, 3001)
    a = -0.37
    fin = wd.upload(psi, prec, parity=1)
    fx = wd.upload(x, prec, parity=0)
    fout = wd.new_field(prec)
    wd.dslash_xpay(fout, fin, fx, a, 0, False, prec)
    got = wd.download(fout, prec, parity=0)
    want = (x + a * oracle.dslash(psi * parity_mask(dims, 1), U, dims, out_parity=0)) * parity_mask(dims, 0)
    assert rel_err(got, want) <= TOL[prec]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("dagger", [False, True])
def test_apply_M_full_and_schur(wdp, prec, dagger):
    dims = (8, 6, 4, 16)
    kappa = 0.124
    wd, U = lattice(dims)
    psi = li.gaussian_spinor(dims, 3100)
    fin = wd.upload(psi, prec)
    fout = wd.new_field(prec, 2)
    wd.apply_M(fout, fin, kappa, wdp.M_FULL, dagger, prec)
    got = wd.download(fout, prec)
    want = oracle.apply_M(psi, U, dims, kappa, dagger=dagger)
    assert rel_err(got, want) <= TOL[prec]
    ev = parity_mask(dims, 0)
    fe = wd.upload(psi, prec, parity=0)
    fo = wd.new_field(prec)
    wd.apply_M(fo, fe, kappa, wdp.M_SCHUR_EVEN, dagger, prec)
    got = wd.download(fo, prec, parity=0)
    want = oracle.apply_Mhat(psi * ev, U, dims, kappa, dagger=dagger)
    assert rel_err(got, want) <= TOL[prec]


@pytest.mark.parametrize("prec,fmt", [(2, oracle.FMT_Q16), (3, oracle.FMT_H16N), (4, oracle.FMT_B16N)])
def test_codec_bitwise(wdp, prec, fmt):
    """Codes and norms written by the GPU equal the oracle's encode bit for bit."""
    dims = (4, 6, 8, 10)
    wd, _ = lattice(dims)
    rng = np.random.default_rng(17)
    psi = li.gaussian_spinor(dims, 3200) * np.exp(rng.uniform(-9, 2, size=(li.volume(dims), 4, 3)))
    psi[parity_sites(dims, 0)[:5]] = 0.0  # zero spinors: norm 0, codes 0
    f = wd.upload(psi, prec, parity=0)
    codes, norms = split16(f.cpu().numpy(), dims)
    sites = parity_sites(dims, 0)
    # the library stores S psi (App. B basis change at the boundary)
    ocodes, ovals, onorms = oracle.encode_spinor(to_internal_basis(psi[sites]), fmt)
    np.testing.assert_array_equal(norms, onorms)
    if fmt == oracle.FMT_Q16:
        np.testing.assert_array_equal(codes.view(np.int16), ocodes)
    elif fmt == oracle.FMT_H16N:
        np.testing.assert_array_equal(codes.view(np.float16).astype(np.float32), ovals)
    else:
        as_f32 = (codes.astype(np.uint32) << 16).view(np.float32)
        np.testing.assert_array_equal(as_f32, ovals)
    # export decodes exactly as the oracle's decode
    got = wd.download(f, prec, parity=0)[sites]
    dec = oracle.decode_spinor(ocodes, ovals, onorms, fmt).view(np.complex128).reshape(-1, 4, 3)
    np.testing.assert_array_equal(got, to_host_basis(dec))


@pytest.mark.parametrize("prec", PRECS)
def test_norm2_fp64_reduction(wdp, prec):
    dims = (8, 8, 8, 16)
    wd, _ = lattice(dims)
    psi = li.gaussian_spinor(dims, 3300)
    f = wd.upload(psi, prec, parity=1)
    stored = wd.download(f, prec, parity=1)
    n = wd.norm2(f, prec)
    assert abs(n - np.vdot(stored, stored).real) <= 1e-12 * n
    assert wd.norm2(f, prec) == n  # fixed-order reduction: bitwise repeatable


def test_f32_export_roundtrip(wdp):
    dims = (4, 4, 4, 4)
    wd, _ = lattice(dims)
    psi = li.gaussian_spinor(dims, 3400)
    f = wd.upload(psi, 1, parity=0)
    got = wd.download(f, 1, parity=0)
    sites = parity_sites(dims, 0)
    internal = to_internal_basis(psi[sites]).astype(np.complex64).astype(np.complex128)
    np.testing.assert_array_equal(got[sites], to_host_basis(internal))


def test_free_field_plane_wave(wdp):
    """Unit links: D psi = sum_mu (2 cos p_mu - 2 i gamma_mu sin p_mu) psi (exact)."""
    dims = (4, 6, 8, 10)
    import paper_0911_3191_gb300 as m
    wd = m.WilsonDirac(dims, t_antiperiodic=True)
    wd.load_gauge(li.unit_gauge(dims))
    x, y, z, t = li.coords(dims)
    p = [2 * np.pi * 1 / 4, 2 * np.pi * 2 / 6, 0.0, 3 * np.pi / 10]
    u = np.arange(12).reshape(4, 3) * (1 + 0.5j)
    psi = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))[:, None, None] * u[None]
    G = [oracle.gamma(m_) for m_ in range(4)]
    Dp = sum(2 * np.cos(p[k]) * np.eye(4) - 2j * np.sin(p[k]) * G[k] for k in range(4))
    want = np.einsum("ab,sbc->sac", Dp, psi) * parity_mask(dims, 0)
    fin = wd.upload(psi, 0, parity=1)
    fout = wd.new_field(0)
    wd.dslash(fout, fin, 0, False, 0)
    got = wd.download(fout, 0, parity=0)
    assert rel_err(got, want) < 1e-14


@pytest.mark.parametrize("prec", PRECS)
def test_accuracy_distribution_delta(wdp, prec):
    """Delta(eps) of Sec. 4.7: the fraction of M_hat output components that
    deviate from the CPU result by >= eps, for uniform eta in [0,1] and
    random SU(3) links; zero beyond the precision's accuracy, one well below."""
    dims = (8, 8, 8, 8)
    kappa = 0.12
    wd, U = lattice(dims, eps=3.0)
    eta = li.uniform_spinor(dims, 3500) * parity_mask(dims, 0)
    f = wd.upload(eta, prec, parity=0)
    o = wd.new_field(prec)
    wd.apply_M(o, f, kappa, wdp.M_SCHUR_EVEN, False, prec)
    got = wd.download(o, prec, parity=0)[parity_sites(dims, 0)].reshape(-1, 12).view(np.float64)
    want = oracle.apply_Mhat(eta, U, dims, kappa)[parity_sites(dims, 0)].reshape(-1, 12).view(np.float64)
    dev = np.abs(got - want).ravel()

    def delta(e):
        return float(np.mean(dev >= e))

    accuracy = {0: 1e-13, 1: 1e-5, 2: 5e-2, 3: 5e-2, 4: 2e-1}[prec]
    assert delta(accuracy) == 0.0
    assert delta(accuracy * 1e-4) > 0.5 or prec == 0
    eps = np.logspace(-17, 0, 35)
    curve = [delta(e) for e in eps]
    assert all(a >= b for a, b in zip(curve, curve[1:]))  # a cumulative distribution
