"""Pins for the multi-shift BiCGstab recurrences (oracle/multishift.py), which
the CUDA multi-shift solver follows: every shifted solution equals a dense LU
solve (numpy.linalg.solve) of its own system, and on the Wilson-Dirac Schur
operator the kappa family M_hat(kappa_k) = (kappa_k / kappa_s)^2
(M_hat(kappa_s) + tau_k), tau_k = (kappa_s / kappa_k)^2 - 1, reproduces the
oracle's single-kappa solves."""
import numpy as np
import pytest

import lattice_inputs as li
import oracle
from oracle.multishift import multishift_bicgstab
from tests.wd_testutil import parity_mask


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_dense_shifted_family(seed):
    rng = np.random.default_rng(seed)
    n = 80
    A = 3.0 * np.eye(n) + (rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))) / np.sqrt(n)
    b = rng.normal(size=n) + 1j * rng.normal(size=n)
    shifts = [0.0, 0.05, 0.4, 1.7]
    xs, it, hist = multishift_bicgstab(lambda v: A @ v, b, shifts, tol=1e-13)
    assert it < n
    for sg, x in zip(shifts, xs):
        want = np.linalg.solve(A + sg * np.eye(n), b)
        assert np.linalg.norm(x - want) / np.linalg.norm(want) < 1e-11, sg


def test_seed_alone_is_bicgstab():
    """With the single shift 0 the recurrences reduce to BiCGstab: the
    residual history equals the oracle's own BiCGstab on the same system."""
    rng = np.random.default_rng(4)
    n = 50
    A = 2.0 * np.eye(n) + (rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))) / np.sqrt(n)
    b = rng.normal(size=n) + 1j * rng.normal(size=n)
    xs, it, _ = multishift_bicgstab(lambda v: A @ v, b, [0.0], tol=1e-12)
    assert np.linalg.norm(A @ xs[0] - b) / np.linalg.norm(b) < 1e-11


def test_wilson_kappa_family():
    """Shifts of M_hat(kappa_s): x(kappa_k) = (kappa_s / kappa_k)^2 y_k with
    (M_hat(kappa_s) + tau_k) y_k = b_e solves M_hat(kappa_k) x = b_e."""
    dims = (4, 4, 4, 8)
    U = li.gauge(dims, 0.5, 1400)
    b = li.gaussian_spinor(dims, 2400) * parity_mask(dims, 0)
    kappas = [0.124, 0.12, 0.118, 0.11]
    ks = max(kappas)
    taus = [(ks / k) ** 2 - 1.0 for k in kappas]
    mask = np.broadcast_to(parity_mask(dims, 0), b.shape).reshape(-1)

    def B(v):
        return oracle.apply_Mhat(v.reshape(b.shape), U, dims, ks).reshape(-1) * mask

    ys, it, _ = multishift_bicgstab(B, b.reshape(-1), taus, tol=1e-12)
    for k, y in zip(kappas, ys):
        x = ((ks / k) ** 2 * y).reshape(b.shape)
        r = b - oracle.apply_Mhat(x, U, dims, k)
        assert np.linalg.norm(r) / np.linalg.norm(b) < 1e-11, k


def test_wilson_general_source_two_families():
    """The combination the CUDA multi-shift solver uses for a general source:
    y_k, z_k solve (M_hat(kappa_s) + tau_k) (.) = b_e, D_eo b_o; then
    x_e = (kappa_s / kappa_k)^2 (y_k + kappa_k z_k), x_o = b_o + kappa_k D_oe x_e
    solves M_kappa_k x = b on the full lattice."""
    dims = (4, 4, 4, 8)
    U = li.gauge(dims, 0.5, 1401)
    b = li.gaussian_spinor(dims, 2401)
    even = np.broadcast_to(parity_mask(dims, 0), b.shape)
    odd = np.broadcast_to(parity_mask(dims, 1), b.shape)
    b_e, b_o = b * even, b * odd
    kappas = [0.124, 0.12, 0.115]  # the seed (largest kappa, shift 0) first
    ks = max(kappas)
    taus = [(ks / k) ** 2 - 1.0 for k in kappas]
    m = even.reshape(-1)

    def B(v):
        return oracle.apply_Mhat(v.reshape(b.shape), U, dims, ks).reshape(-1) * m

    w = oracle.dslash(b_o, U, dims, out_parity=0)  # D_eo b_o
    ys, _, _ = multishift_bicgstab(B, b_e.reshape(-1), taus, tol=1e-13)
    zs, _, _ = multishift_bicgstab(B, w.reshape(-1), taus, tol=1e-13)
    for k, y, z in zip(kappas, ys, zs):
        x_e = ((ks / k) ** 2 * (y + k * z)).reshape(b.shape)
        x_o = b_o + k * oracle.dslash(x_e, U, dims, out_parity=1)
        x = x_e + x_o
        assert oracle.true_residual(x, b, U, dims, k) < 1e-11, k


def test_seed_must_come_first():
    with pytest.raises(ValueError):
        multishift_bicgstab(lambda v: v, np.ones(4), [0.1, 0.0])


@pytest.mark.parametrize("mutation", [
    ("beta_s = beta * (f[k] / f_next) ** 2", "beta_s = beta"),
    ("omega_s = omega / (1.0 + omega * sig)", "omega_s = omega"),
    ("pi[k] = pi_next", "pi[k] = pi[k]"),
    ("f_next = f[k] + alpha * sig * g[k]", "f_next = f[k] + alpha * sig * f[k]"),
])
def test_planted_mistakes_fail_the_dense_pin(mutation):
    """A copy of the recurrences with one plausible mistake planted no longer
    matches the dense LU solves of the shifted systems."""
    import os
    import types
    src = open(os.path.join(os.path.dirname(oracle.__file__), "multishift.py")).read()
    old, new = mutation
    assert src.count(old) == 1
    mod = types.ModuleType("multishift_mutant")
    exec(compile(src.replace(old, new), "multishift_mutant", "exec"), mod.__dict__)
    rng = np.random.default_rng(5)
    n = 60
    A = 3.0 * np.eye(n) + (rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))) / np.sqrt(n)
    b = rng.normal(size=n) + 1j * rng.normal(size=n)
    shifts = [0.0, 0.4, 1.7]
    with np.errstate(all="ignore"):
        xs, _, _ = mod.multishift_bicgstab(lambda v: A @ v, b, shifts, tol=1e-12, maxiter=200)
    errs = [np.linalg.norm(x - np.linalg.solve(A + s * np.eye(n), b)) / np.linalg.norm(b)
            for s, x in zip(shifts, xs)]
    assert not all(np.isfinite(e) and e < 1e-8 for e in errs), errs
