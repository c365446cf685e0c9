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
