"""Pins for the CPU oracle (arXiv:0911.3191), checked against what the paper
and the mathematics fix -- never against the oracle's own formulas:

* the DeGrand-Rossi projectors printed in App. B and the Clifford algebra;
* the free-field (unit-link) plane-wave closed form of D, M and M_hat and the
  exact solution of M x = b for a plane-wave source (Sec. 3 matrix);
* D^dag is the adjoint of D; gamma_5-hermiticity of M and M_hat;
* gauge covariance under a random SU(3) transformation;
* M_hat equals the Schur complement of the dense M (Sec. 3), and the solvers
  agree with a dense LU solve (numpy.linalg.solve) on a 4^4 lattice;
* the 16-bit codecs: exact maximum, error bound, fp16 and bf16 rounding
  against numpy's float16 and torch's bfloat16 conversions.
"""
import numpy as np
import pytest

import lattice_inputs as li
import oracle

# App. B, DeGrand-Rossi basis: P^{+mu} = 1 + gamma_mu (upper signs as printed)
J = 1j
P_PLUS_PRINTED = [
    np.array([[1, 0, 0, J], [0, 1, J, 0], [0, -J, 1, 0], [-J, 0, 0, 1]]),
    np.array([[1, 0, 0, -1], [0, 1, 1, 0], [0, 1, 1, 0], [-1, 0, 0, 1]]),
    np.array([[1, 0, J, 0], [0, 1, 0, -J], [-J, 0, 1, 0], [0, J, 0, 1]]),
    np.array([[1, 0, 1, 0], [0, 1, 0, 1], [1, 0, 1, 0], [0, 1, 0, 1]]),
]
# lower signs as printed: P^{-mu}
P_MINUS_PRINTED = [
    np.array([[1, 0, 0, -J], [0, 1, -J, 0], [0, J, 1, 0], [J, 0, 0, 1]]),
    np.array([[1, 0, 0, 1], [0, 1, -1, 0], [0, -1, 1, 0], [1, 0, 0, 1]]),
    np.array([[1, 0, -J, 0], [0, 1, 0, J], [J, 0, 1, 0], [0, -J, 0, 1]]),
    np.array([[1, 0, -1, 0], [0, 1, 0, -1], [-1, 0, 1, 0], [0, -1, 0, 1]]),
]
G = [P_PLUS_PRINTED[m] - np.eye(4) for m in range(4)]
G5 = G[0] @ G[1] @ G[2] @ G[3]


def spin_apply(mat, psi):
    """Apply a 4x4 spin matrix to a (V, 4, 3) field."""
    return np.einsum("ab,sbc->sac", mat, psi)


def inner(a, b):
    return np.vdot(a.ravel(), b.ravel())


# ------------------------------------------------------------------ gammas
def test_gamma_matches_printed_projectors():
    for mu in range(4):
        g = oracle.gamma(mu)
        np.testing.assert_array_equal(g, G[mu])
        np.testing.assert_array_equal(np.eye(4) - g, P_MINUS_PRINTED[mu])


def test_clifford_algebra_and_gamma5():
    for mu in range(4):
        assert np.allclose(G[mu], G[mu].conj().T)
        for nu in range(4):
            ac = G[mu] @ G[nu] + G[nu] @ G[mu]
            assert np.allclose(ac, 2 * np.eye(4) * (mu == nu))
        assert np.allclose(G5 @ G[mu] + G[mu] @ G5, 0)
    assert np.allclose(G5 @ G5, np.eye(4))
    assert np.allclose(G5, G5.conj().T)
    # App. B calls DeGrand-Rossi a chiral basis: gamma_5 is diagonal there
    assert np.allclose(G5, np.diag(np.diag(G5)))


def test_projectors_rank_two():
    for mu in range(4):
        for P in (P_PLUS_PRINTED[mu], P_MINUS_PRINTED[mu]):
            assert np.allclose(P @ P, 2 * P)
            assert np.linalg.matrix_rank(P) == 2


# ------------------------------------------------------------ free field
def plane_wave(dims, n, u, anti=False):
    """psi(x) = exp(i p.x) u, p_mu = 2 pi n_mu / L_mu ((2n+1) pi / T in t if antiperiodic)."""
    x, y, z, t = li.coords(dims)
    p = [2 * np.pi * n[m] / dims[m] for m in range(4)]
    if anti:
        p[3] = (2 * n[3] + 1) * np.pi / dims[3]
    phase = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
    return phase[:, None, None] * u[None, :, :], p


def d_of_p(p, dagger=False):
    s = 1.0 if dagger else -1.0
    return sum(2 * np.cos(p[m]) * np.eye(4) + s * 2j * np.sin(p[m]) * G[m] for m in range(4))


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (4, 6, 8, 10)])
@pytest.mark.parametrize("n", [(0, 0, 0, 0), (1, 0, 0, 0), (0, 1, 2, 3), (1, 2, 3, 1)])
@pytest.mark.parametrize("dagger", [False, True])
@pytest.mark.parametrize("anti", [False, True])
def test_free_field_dslash_closed_form(dims, n, dagger, anti):
    rng = np.random.default_rng(7)
    u = rng.normal(size=(4, 3)) + 1j * rng.normal(size=(4, 3))
    psi, p = plane_wave(dims, n, u, anti)
    U = li.unit_gauge(dims)
    got = oracle.dslash(psi, U, dims, dagger=dagger, tbc_anti=anti)
    want = spin_apply(d_of_p(p, dagger), psi)
    assert np.abs(got - want).max() < 1e-12


@pytest.mark.parametrize("n", [(0, 0, 0, 0), (1, 2, 0, 3)])
@pytest.mark.parametrize("anti", [False, True])
def test_free_field_mhat_closed_form(n, anti):
    dims = (4, 6, 4, 8)
    kappa = 0.11
    rng = np.random.default_rng(3)
    u = rng.normal(size=(4, 3)) + 1j * rng.normal(size=(4, 3))
    psi, p = plane_wave(dims, n, u, anti)
    even = (li.parity(dims) == 0)[:, None, None]
    psi_e = psi * even
    got = oracle.apply_Mhat(psi_e, li.unit_gauge(dims), dims, kappa, tbc_anti=anti)
    Dp = d_of_p(p)
    want = spin_apply(np.eye(4) - kappa ** 2 * Dp @ Dp, psi) * even
    assert np.abs(got - want).max() < 1e-12
    got_m = oracle.apply_M(psi, li.unit_gauge(dims), dims, kappa, tbc_anti=anti)
    assert np.abs(got_m - spin_apply(np.eye(4) - kappa * Dp, psi)).max() < 1e-12


@pytest.mark.parametrize("solver,schur", [("bicgstab", True), ("bicgstab", False), ("cgnr", True)])
def test_free_field_exact_solution(solver, schur):
    dims = (4, 4, 6, 8)
    kappa = 0.12
    rng = np.random.default_rng(11)
    u = rng.normal(size=(4, 3)) + 1j * rng.normal(size=(4, 3))
    b, p = plane_wave(dims, (1, 0, 2, 3), u, anti=True)
    x_exact = spin_apply(np.linalg.inv(np.eye(4) - kappa * d_of_p(p)), b)
    x, st, iters, rel = oracle.solve(b, li.unit_gauge(dims), dims, kappa, tol=1e-12, solver=solver,
                                     schur=schur, tbc_anti=True)
    assert st == 0 and rel <= 1e-12 and iters > 0
    assert np.linalg.norm(x - x_exact) / np.linalg.norm(x_exact) < 1e-10


# ------------------------------------------------- adjoint, gamma5, gauge
@pytest.fixture(scope="module")
def rand_lattice():
    dims = (4, 6, 4, 8)
    U = li.gauge(dims, 0.5, 1001)
    phi = li.gaussian_spinor(dims, 2001)
    psi = li.gaussian_spinor(dims, 2002)
    return dims, U, phi, psi


@pytest.mark.parametrize("anti", [False, True])
def test_dagger_is_adjoint(rand_lattice, anti):
    dims, U, phi, psi = rand_lattice
    lhs = inner(phi, oracle.dslash(psi, U, dims, tbc_anti=anti))
    rhs = inner(oracle.dslash(phi, U, dims, dagger=True, tbc_anti=anti), psi)
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)


@pytest.mark.parametrize("anti", [False, True])
def test_gamma5_hermiticity(rand_lattice, anti):
    dims, U, phi, psi = rand_lattice
    kappa = 0.12
    # D^dag = gamma5 D gamma5
    a = oracle.dslash(psi, U, dims, dagger=True, tbc_anti=anti)
    b = spin_apply(G5, oracle.dslash(spin_apply(G5, psi), U, dims, tbc_anti=anti))
    assert np.abs(a - b).max() < 1e-12
    # <phi, gamma5 M gamma5 psi> = <M phi, psi>
    lhs = inner(phi, spin_apply(G5, oracle.apply_M(spin_apply(G5, psi), U, dims, kappa, tbc_anti=anti)))
    rhs = inner(oracle.apply_M(phi, U, dims, kappa, tbc_anti=anti), psi)
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)
    # the same for M_hat on even sites, and its dagger flag
    even = (li.parity(dims) == 0)[:, None, None]
    pe, qe = phi * even, psi * even
    lhs = inner(pe, oracle.apply_Mhat(qe, U, dims, kappa, tbc_anti=anti))
    rhs = inner(oracle.apply_Mhat(pe, U, dims, kappa, dagger=True, tbc_anti=anti), qe)
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)
    g5m = spin_apply(G5, oracle.apply_Mhat(spin_apply(G5, qe), U, dims, kappa, tbc_anti=anti))
    assert np.abs(g5m - oracle.apply_Mhat(qe, U, dims, kappa, dagger=True, tbc_anti=anti)).max() < 1e-12


@pytest.mark.parametrize("anti", [False, True])
def test_gauge_covariance(rand_lattice, anti):
    dims, U, _, psi = rand_lattice
    V = li.volume(dims)
    Gx = li.su3_field(V, 3.0, 4242)
    x, y, z, t = li.coords(dims)
    Up = np.empty_like(U)
    for mu in range(4):
        c = [x, y, z, t]
        c[mu] = (c[mu] + 1) % dims[mu]
        fwd = li.lex_index(dims, *c)
        Up[:, mu] = Gx @ U[:, mu] @ Gx[fwd].conj().transpose(0, 2, 1)
    psip = np.einsum("sij,saj->sai", Gx, psi)
    got = oracle.dslash(psip, Up, dims, tbc_anti=anti)
    want = np.einsum("sij,saj->sai", Gx, oracle.dslash(psi, U, dims, tbc_anti=anti))
    assert np.abs(got - want).max() < 1e-12


# ------------------------------------------------- dense 4^4 brute force
@pytest.fixture(scope="module")
def dense_4x4():
    dims = (4, 4, 4, 4)
    kappa = 0.12
    U = li.gauge(dims, 0.5, 1000)
    V = li.volume(dims)
    n = 12 * V
    M = np.empty((n, n), dtype=np.complex128)
    e = np.zeros(n, dtype=np.complex128)
    for j in range(n):
        e[j] = 1.0
        M[:, j] = oracle.apply_M(e.reshape(V, 4, 3), U, dims, kappa).ravel()
        e[j] = 0.0
    return dims, kappa, U, M


def test_dense_dagger(dense_4x4):
    dims, kappa, U, M = dense_4x4
    V = li.volume(dims)
    rng = np.random.default_rng(5)
    v = rng.normal(size=(V, 4, 3)) + 1j * rng.normal(size=(V, 4, 3))
    got = oracle.apply_M(v, U, dims, kappa, dagger=True).ravel()
    assert np.abs(got - M.conj().T @ v.ravel()).max() < 1e-12


def test_dense_schur_complement(dense_4x4):
    dims, kappa, U, M = dense_4x4
    V = li.volume(dims)
    par = np.repeat(li.parity(dims), 12)
    e_idx, o_idx = np.where(par == 0)[0], np.where(par == 1)[0]
    Mee, Meo = M[np.ix_(e_idx, e_idx)], M[np.ix_(e_idx, o_idx)]
    Moe, Moo = M[np.ix_(o_idx, e_idx)], M[np.ix_(o_idx, o_idx)]
    S = Mee - Meo @ np.linalg.solve(Moo, Moe)
    rng = np.random.default_rng(6)
    for _ in range(3):
        v = np.zeros(12 * V, dtype=np.complex128)
        v[e_idx] = rng.normal(size=len(e_idx)) + 1j * rng.normal(size=len(e_idx))
        got = oracle.apply_Mhat(v.reshape(V, 4, 3), U, dims, kappa).ravel()
        assert np.abs(got[e_idx] - S @ v[e_idx]).max() < 1e-12
        assert np.abs(got[o_idx]).max() == 0.0


@pytest.mark.parametrize("solver,schur", [("bicgstab", True), ("bicgstab", False), ("cgnr", True),
                                          ("cgnr", False)])
def test_dense_solve(dense_4x4, solver, schur):
    dims, kappa, U, M = dense_4x4
    V = li.volume(dims)
    b = li.gaussian_spinor(dims, 2100)
    x_ref = np.linalg.solve(M, b.ravel())
    x, st, iters, rel = oracle.solve(b, U, dims, kappa, tol=1e-12, solver=solver, schur=schur)
    assert st == 0 and rel <= 1e-12
    assert np.linalg.norm(x.ravel() - x_ref) / np.linalg.norm(x_ref) < 1e-10
    r = b.ravel() - M @ x.ravel()
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 1e-12
    if schur:
        # odd rows of the full residual vanish once x_o is reconstructed
        par = np.repeat(li.parity(dims), 12)
        assert np.abs(r[par == 1]).max() < 1e-13 * np.abs(b).max() * 10


def test_schur_residual_equals_full_residual(rand_lattice):
    """|b - M x| = |b_hat - M_hat x_e| for any x_e when x_o is reconstructed."""
    dims, U, phi, b = rand_lattice
    kappa = 0.124
    even = (li.parity(dims) == 0)[:, None, None]
    xe = phi * even
    b_hat = (b + kappa * oracle.dslash(b * ~even, U, dims, out_parity=0)) * even
    x = xe + (b + kappa * oracle.dslash(xe, U, dims, out_parity=1)) * ~even
    full = b - oracle.apply_M(x, U, dims, kappa)
    schur = b_hat - oracle.apply_Mhat(xe, U, dims, kappa)
    assert np.abs(full[~even[:, 0, 0]]).max() < 1e-13
    assert abs(np.linalg.norm(full) - np.linalg.norm(schur)) < 1e-12 * np.linalg.norm(full)


# ------------------------------------------------------------ codecs
def _spinors(n, seed):
    rng = np.random.default_rng(seed)
    v = rng.normal(size=(n, 12)) + 1j * rng.normal(size=(n, 12))
    # widen the dynamic range inside a site so small elements (and fp16
    # subnormals after normalisation) occur
    v *= np.exp(rng.uniform(-12, 2, size=(n, 12)))
    return v


def test_q16_codec_bounds():
    v = _spinors(2000, 1)
    codes, _, norms = oracle.encode_spinor(v, oracle.FMT_Q16)
    f = v.view(np.float64).reshape(-1, 24).astype(np.float32)
    np.testing.assert_array_equal(norms, np.abs(f).max(axis=1))
    assert np.abs(codes.astype(np.int32)).max() <= 32767
    # the element that defines the norm is stored as exactly +-32767
    imax = np.abs(f).argmax(axis=1)
    assert np.all(np.abs(codes[np.arange(len(codes)), imax]) == 32767)
    dec = oracle.decode_spinor(codes, None, norms, oracle.FMT_Q16)
    err = np.abs(dec - f.astype(np.float64))
    assert np.all(err <= norms[:, None] * (1.0 / 65534 + 1e-6))
    z, _, zn = oracle.encode_spinor(np.zeros((3, 12), np.complex128), oracle.FMT_Q16)
    assert np.all(z == 0) and np.all(zn == 0)


@pytest.mark.parametrize("fmt", [oracle.FMT_H16N, oracle.FMT_B16N])
def test_float16_codecs_against_library_rounding(fmt):
    torch = pytest.importorskip("torch")
    v = _spinors(2000, 2)
    _, vals, norms = oracle.encode_spinor(v, fmt)
    f = v.view(np.float64).reshape(-1, 24).astype(np.float32)
    w = f * (np.float32(1.0) / norms[:, None])
    assert w.dtype == np.float32
    if fmt == oracle.FMT_H16N:
        want = w.astype(np.float16).astype(np.float32)
    else:
        want = torch.from_numpy(w).to(torch.bfloat16).to(torch.float32).numpy()
    np.testing.assert_array_equal(vals, want)
    if fmt == oracle.FMT_H16N:
        assert np.any((np.abs(want) < 6.1e-5) & (want != 0))  # subnormals exercised


def test_link_codecs():
    torch = pytest.importorskip("torch")
    U = li.gauge((2, 2, 2, 2), 0.7, 9).view(np.float64).ravel()
    codes, dec = oracle.encode_link_values(U, oracle.FMT_Q16)
    assert np.abs(dec - U).max() <= 1.0 / 65534 + 1e-7
    np.testing.assert_array_equal(codes, np.rint(U.astype(np.float32) * np.float32(32767)).astype(np.int16))
    _, dh = oracle.encode_link_values(U, oracle.FMT_H16N)
    np.testing.assert_array_equal(dh, U.astype(np.float32).astype(np.float16).astype(np.float64))
    _, db = oracle.encode_link_values(U, oracle.FMT_B16N)
    want = torch.from_numpy(U.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(db, want)


# ------------------------------------------------------------ inputs
def test_philox_known_answers():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(h, 16) for h in r]
        assert li.philox4x32_10(v[0:4], v[4:6]) == tuple(v[6:10])


def test_generated_links_are_su3_with_third_row_from_first_two():
    U = li.gauge((4, 4, 4, 8), 0.3, 1002).reshape(-1, 3, 3)
    assert np.abs(U @ U.conj().transpose(0, 2, 1) - np.eye(3)).max() < 1e-14
    assert np.abs(np.linalg.det(U) - 1).max() < 1e-14
    c = np.conj(np.cross(U[:, 0], U[:, 1]))
    assert np.abs(c - U[:, 2]).max() < 1e-14
    # eps controls the distance from the unit matrix
    U2 = li.gauge((4, 4, 4, 8), 0.05, 1002).reshape(-1, 3, 3)
    assert np.abs(U2 - np.eye(3)).mean() < np.abs(U - np.eye(3)).mean()


# ---- App. A.2: the 8-number parametrisation
@pytest.mark.parametrize("eps", [0.3, 1.0, 3.0])
def test_su3_8number_roundtrip(eps):
    """Encoding a link into (arg a1, arg c1, a2, a3, b1) and rebuilding it
    gives the link back (away from the singularity |a1| = 1)."""
    U = li.su3_field(500, eps, 77).reshape(-1, 3, 3)
    p, sing = oracle.su3_to8(U)
    assert not sing.any()
    N = np.sqrt(np.abs(U[:, 0, 1]) ** 2 + np.abs(U[:, 0, 2]) ** 2)
    err = np.abs(oracle.su3_from8(p) - U).max(axis=(1, 2))
    assert np.all(err <= 1e-14 / N)


def test_su3_8number_rebuilds_su3_from_any_valid_parameters():
    """Any parameters in the valid region give a special unitary matrix whose
    stored entries are the given ones (|a1|, |c1| from unit row / column)."""
    rng = np.random.default_rng(3)
    for _ in range(200):
        a2, a3 = (rng.normal(size=2) @ [1, 1j]) * 0.5, (rng.normal(size=2) @ [1, 1j]) * 0.5
        s = abs(a2) ** 2 + abs(a3) ** 2
        if s >= 0.99:
            continue
        b1 = (rng.normal(size=2) @ [1, 1j])
        b1 *= rng.uniform(0, 1) * np.sqrt(s) / abs(b1)  # |b1|^2 <= 1 - |a1|^2 = s
        p = np.array([rng.uniform(-np.pi, np.pi), rng.uniform(-np.pi, np.pi), a2.real, a2.imag, a3.real, a3.imag,
                      b1.real, b1.imag])
        U = oracle.su3_from8(p)
        np.testing.assert_allclose(U @ U.conj().T, np.eye(3), atol=1e-13)
        assert abs(np.linalg.det(U) - 1) < 1e-13
        assert abs(U[0, 1] - a2) < 1e-15 and abs(U[0, 2] - a3) < 1e-15 and abs(U[1, 0] - b1) < 1e-15
        assert abs(np.angle(U[0, 0]) - p[0]) % (2 * np.pi) < 1e-12 or abs(U[0, 0]) < 1e-12


def test_su3_8number_singularity_flagged():
    assert oracle.su3_to8(np.eye(3, dtype=np.complex128))[1]
    D = np.diag(np.exp(1j * np.array([0.3, -0.5, 0.2])))
    assert oracle.su3_to8(D)[1]


@pytest.mark.parametrize("anti", [False, True])
def test_temporal_gauge_reading(rand_lattice, anti):
    """The temporal-gauge transformation as read from Sec. 4.3:
    G(x, 0) = 1, G(x, t+1) = G(x, t) U_4(x, t).  The transformed temporal
    links are the unit matrix off the last time slice, the last slice holds
    the product of U_4 around the time direction (gauge-invariant trace), and
    the operator transforms covariantly, D[U'] G psi = G D[U] psi."""
    dims, U, _, psi = rand_lattice
    X, Y, Z, T = dims
    ns = X * Y * Z
    V = li.volume(dims)
    U4 = U.reshape(T, ns, 4, 3, 3)[:, :, 3]
    G = np.empty((T, ns, 3, 3), dtype=np.complex128)
    G[0] = np.eye(3)
    for t in range(1, T):
        G[t] = G[t - 1] @ U4[t - 1]
    G = G.reshape(V, 3, 3)
    x, y, z, t = li.coords(dims)
    Up = np.empty_like(U)
    for mu in range(4):
        c = [x, y, z, t]
        c[mu] = (c[mu] + 1) % dims[mu]
        fwd = li.lex_index(dims, *c)
        Up[:, mu] = G @ U[:, mu] @ G[fwd].conj().transpose(0, 2, 1)
    last = (t == T - 1)
    assert np.abs(Up[~last, 3] - np.eye(3)).max() < 1e-13
    # on the last slice: the ordered product U_4(x,0) ... U_4(x,T-1)
    prod = np.broadcast_to(np.eye(3), (ns, 3, 3)).copy()
    for tt in range(T):
        prod = prod @ U4[tt]
    assert np.abs(Up[last, 3] - prod).max() < 1e-12
    psip = np.einsum("sij,saj->sai", G, psi)
    got = oracle.dslash(psip, Up, dims, tbc_anti=anti)
    want = np.einsum("sij,saj->sai", G, oracle.dslash(psi, U, dims, tbc_anti=anti))
    assert np.abs(got - want).max() < 1e-12


# ---- D at a list of sites (the checker of the full-size GPU parity tests)
def _boundary_sites(dims, rng, n_random=200):
    """Every combination of {0, 1, middle, L-2, L-1} per direction (all corner,
    edge and face patterns of the boundary, both parities), random sites, and
    duplicates in shuffled order."""
    picks = [sorted({0, 1, d // 2, d - 2, d - 1}) for d in dims]
    grid = np.stack(np.meshgrid(*picks, indexing="ij"), axis=-1).reshape(-1, 4)
    lex = li.lex_index(dims, grid[:, 0], grid[:, 1], grid[:, 2], grid[:, 3])
    rnd = rng.integers(0, li.volume(dims), size=n_random)
    sites = np.concatenate([lex, rnd, lex[::7], rnd[:17]])
    rng.shuffle(sites)
    return sites.astype(np.int64)


@pytest.mark.parametrize("dims", [(4, 6, 8, 10), (6, 4, 2, 12)])
@pytest.mark.parametrize("dagger", [False, True])
@pytest.mark.parametrize("anti", [False, True])
def test_dslash_sites_equals_full_lattice_dslash(dims, dagger, anti):
    """D psi at a list of sites equals the (pinned) full-lattice D psi at those
    sites, bit for bit, for both parities, with duplicated and unordered
    entries in the list."""
    rng = np.random.default_rng(31)
    U = li.gauge(dims, 0.5, 1011)
    psi = li.gaussian_spinor(dims, 2011)
    sites = _boundary_sites(dims, rng)
    got = oracle.dslash_sites(psi, U, dims, sites, dagger=dagger, tbc_anti=anti)
    full = oracle.dslash(psi, U, dims, dagger=dagger, tbc_anti=anti)
    np.testing.assert_array_equal(got, full[sites])
    par = li.parity(dims)[sites]
    for p in (0, 1):
        one = oracle.dslash(psi, U, dims, dagger=dagger, out_parity=p, tbc_anti=anti)
        np.testing.assert_array_equal(got[par == p], one[sites[par == p]])
    assert set(par.tolist()) == {0, 1}


@pytest.mark.parametrize("dims", [(4, 6, 8, 10), (6, 4, 2, 12)])
@pytest.mark.parametrize("dagger", [False, True])
@pytest.mark.parametrize("anti", [False, True])
def test_dslash_sites_free_field_closed_form(dims, dagger, anti):
    """D psi at listed sites against the plane-wave closed form
    D(p) = sum_mu (2 cos p_mu -+ 2 i gamma_mu sin p_mu), independently of the
    full-lattice operator."""
    rng = np.random.default_rng(32)
    u = rng.normal(size=(4, 3)) + 1j * rng.normal(size=(4, 3))
    psi, p = plane_wave(dims, (1, 1, 1, 2), u, anti)
    sites = _boundary_sites(dims, rng)
    got = oracle.dslash_sites(psi, li.unit_gauge(dims), dims, sites, dagger=dagger, tbc_anti=anti)
    want = spin_apply(d_of_p(p, dagger), psi[sites])
    assert np.abs(got - want).max() < 1e-12


# ---- a fixed number of Schur BiCGstab iterations (the timed CPU baseline)
@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (4, 6, 4, 8)])
@pytest.mark.parametrize("n", [1, 2, 3, 5, 8])
def test_bicgstab_schur_iterations_equal_truncated_solve(dims, n):
    """n iterations on the even part of b leave the residual |b_e - M_hat x_e|
    that the (pinned) Schur solve reports after the same n iterations: with
    b_o = 0, b_hat = b_e and the full residual equals the Schur residual."""
    kappa = 0.124
    U = li.gauge(dims, 0.5, 1012)
    b = li.gaussian_spinor(dims, 2012) * (li.parity(dims) == 0)[:, None, None]
    got = oracle.bicgstab_schur_iterations(b, U, dims, kappa, n)
    _, st, iters, rel = oracle.solve(b, U, dims, kappa, tol=1e-300, maxiter=n, solver="bicgstab", schur=True)
    assert st == 1 and iters == n
    want = rel * np.linalg.norm(b)
    assert abs(got - want) <= 1e-12 * want


def test_bicgstab_schur_iterations_free_field():
    """Closed form on the free field.  For an even plane wave, M_hat acts as the
    4x4 spin matrix A = 1 - kappa^2 D(p)^2, which has exactly two distinct
    eigenvalues (D(p)^2 = a^2 - |b|^2 - 2 i a (b.gamma), (b.gamma)^2 = |b|^2).
    Two BiCGstab iterations contain two BiCG steps, which end with a zero
    residual for such an operator.  After one iteration the residual is the
    BiCG step's s = r - alpha A r, alpha = <r, r> / <r, A r>, minimised over
    omega along A s."""
    dims = (4, 6, 4, 8)
    kappa = 0.124
    rng = np.random.default_rng(33)
    u = rng.normal(size=(4, 3)) + 1j * rng.normal(size=(4, 3))
    psi, p = plane_wave(dims, (1, 1, 0, 3), u)
    even = (li.parity(dims) == 0)[:, None, None]
    b = psi * even
    Dp = d_of_p(p)
    A = np.eye(4) - kappa ** 2 * Dp @ Dp
    assert len(set(np.round(np.linalg.eigvals(A), 10))) == 2
    U = li.unit_gauge(dims)
    bn = np.linalg.norm(b)
    # one iteration: every even site carries the same spin-colour vector up to a phase
    nsite = int(even.sum())
    Au = A @ u
    alpha = np.vdot(u, u) / np.vdot(u, Au)
    s = u - alpha * Au
    As = A @ s
    omega = np.vdot(As, s) / np.vdot(As, As)
    r1 = np.linalg.norm(s - omega * As) * np.sqrt(nsite)
    got1 = oracle.bicgstab_schur_iterations(b, U, dims, kappa, 1)
    assert abs(got1 - r1) <= 1e-12 * bn and r1 > 1e-3 * bn
    got2 = oracle.bicgstab_schur_iterations(b, U, dims, kappa, 2)
    assert got2 <= 1e-12 * bn
