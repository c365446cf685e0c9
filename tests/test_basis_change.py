"""The spin-basis change applied at the host boundary (App. B): S maps the
DeGrand-Rossi gamma matrices onto the "non-relativistic" (UKQCD) ones, both
read off the projectors printed in App. B; in the latter gamma_4 is diagonal,
so temporal hops need half a spinor."""
import numpy as np

from tests.test_oracle_pins import P_PLUS_PRINTED as P_DR
from tests.wd_testutil import S_MATRIX, to_host_basis, to_internal_basis

J = 1j
P_UK = [  # App. B, UKQCD basis, upper signs (P^{+mu})
    np.array([[1, 0, 0, J], [0, 1, J, 0], [0, -J, 1, 0], [-J, 0, 0, 1]]),
    np.array([[1, 0, 0, 1], [0, 1, -1, 0], [0, -1, 1, 0], [1, 0, 0, 1]]),
    np.array([[1, 0, J, 0], [0, 1, 0, -J], [-J, 0, 1, 0], [0, J, 0, 1]]),
    np.diag([2, 2, 0, 0]).astype(complex),
]
P_UK_MINUS4 = np.diag([0, 0, 2, 2]).astype(complex)


def test_S_maps_degrand_rossi_to_ukqcd():
    S = S_MATRIX
    assert np.allclose(S @ S.T, np.eye(4))
    for mu in range(4):
        g_dr = P_DR[mu] - np.eye(4)
        g_uk = P_UK[mu] - np.eye(4)
        assert np.allclose(S @ g_dr @ S.T, g_uk), mu
    assert np.allclose(np.eye(4) - (P_UK[3] - np.eye(4)), P_UK_MINUS4)


def test_basis_helpers_are_S_and_its_transpose():
    rng = np.random.default_rng(3)
    psi = rng.normal(size=(10, 4, 3)) + 1j * rng.normal(size=(10, 4, 3))
    v = to_internal_basis(psi)
    assert np.allclose(v, np.einsum("ab,sbc->sac", S_MATRIX, psi))
    assert np.allclose(to_host_basis(v), psi)
