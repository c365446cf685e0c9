"""Shared helpers of the GPU parity tests (no arithmetic of the method)."""
import numpy as np

import lattice_inputs as li

# Relative L2 tolerances of one dslash against the FP64 oracle on unquantised
# FP64 inputs (the total error, input rounding included).
TOL = {0: 1e-13, 1: 1e-6, 2: 5e-3, 3: 5e-3, 4: 5e-3}


def parity_mask(dims, p):
    return (li.parity(dims) == p)[:, None, None]


def parity_sites(dims, p):
    """Lexicographic sites of parity p in even-odd (field) order."""
    return np.where(li.parity(dims) == p)[0]


def rel_err(got, want):
    return float(np.linalg.norm(got - want) / np.linalg.norm(want))


def stride_of(dims):
    vh = li.volume(dims) // 2
    return (vh + 31) // 32 * 32


def align256(n):
    return (n + 255) & ~255


def split16(raw: np.ndarray, dims):
    """Raw bytes of a 16-bit single-parity field -> (codes uint16 (Vh, 24), norms float32 (Vh,))."""
    vh = li.volume(dims) // 2
    st = stride_of(dims)
    codes = raw[: 48 * st].view(np.uint16).reshape(3, st, 8)[:, :vh, :].transpose(1, 0, 2).reshape(vh, 24)
    off = align256(48 * st)
    norms = raw[off: off + 4 * vh].view(np.float32)
    return codes, norms


# App. B basis change used inside the library: psi_int = S psi_DR, S real
# orthogonal (pinned against the printed projector sets in test_basis_change.py).
R2 = 0.70710678118654752440


def to_internal_basis(psi):
    """(V, 4, 3) DeGrand-Rossi -> internal basis, in the library's operation order."""
    p = np.asarray(psi)
    out = np.empty_like(p)
    out[:, 0] = R2 * (p[:, 1] + p[:, 3])
    out[:, 1] = -R2 * (p[:, 0] + p[:, 2])
    out[:, 2] = R2 * (p[:, 1] - p[:, 3])
    out[:, 3] = R2 * (p[:, 2] - p[:, 0])
    return out


def to_host_basis(v):
    u = np.asarray(v)
    out = np.empty_like(u)
    out[:, 0] = -R2 * (u[:, 1] + u[:, 3])
    out[:, 1] = R2 * (u[:, 0] + u[:, 2])
    out[:, 2] = R2 * (u[:, 3] - u[:, 1])
    out[:, 3] = R2 * (u[:, 0] - u[:, 2])
    return out


S_MATRIX = R2 * np.array([[0, 1, 0, 1], [-1, 0, -1, 0], [0, 1, 0, -1], [-1, 0, 1, 0]], dtype=np.float64)
