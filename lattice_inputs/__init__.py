"""Seeded synthetic inputs (gauge links, sources) shared by the oracle and the
CUDA path.

Holds no arithmetic of the Wilson-Dirac method: it draws Philox4x32-10 random
numbers (Salmon et al., SC'11) and builds SU(3) links U = exp(i eps H) from a
Gaussian traceless Hermitian H, complex-Gaussian spinors, uniform spinors and
point sources.  Every array is FP64 in the host conventions used throughout:

* gauge  : ``(V, 4, 3, 3)`` complex128, site lexicographic ``x + X(y + Y(z + Z t))``,
  ``U[x, mu]`` the link from x to x + mu (mu = 0..3 for x, y, z, t)
* spinor : ``(V, 4, 3)`` complex128, ``[site][spin][colour]``
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_LIB = os.path.join(_HERE, "_lattice_inputs.so")
_lock = threading.Lock()
_lib = None

TAG_GAUGE = 0x67617567
TAG_SPINOR = 0x73706E72
TAG_UNIFORM = 0x756E6966
TAG_TRANSFORM = 0x7866726D


def build(force: bool = False) -> str:
    """Compile ``gen.c`` into a shared library beside it (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            lib.li_su3_field.argtypes = [dp, ctypes.c_int64, ctypes.c_double, ctypes.c_uint64, ctypes.c_uint32]
            lib.li_gaussian.argtypes = [dp, ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint32]
            lib.li_uniform.argtypes = [dp, ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint32]
            u32p = ctypes.POINTER(ctypes.c_uint32)
            lib.li_philox4x32_10.argtypes = [u32p, u32p, u32p]
            for f in (lib.li_su3_field, lib.li_gaussian, lib.li_uniform, lib.li_philox4x32_10):
                f.restype = None
            _lib = lib
    return _lib


def _dptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def volume(dims) -> int:
    x, y, z, t = (int(d) for d in dims)
    return x * y * z * t


def philox4x32_10(ctr, key) -> tuple:
    """One raw Philox4x32-10 block (for known-answer tests)."""
    lib = _load()
    c = (ctypes.c_uint32 * 4)(*ctr)
    k = (ctypes.c_uint32 * 2)(*key)
    o = (ctypes.c_uint32 * 4)()
    lib.li_philox4x32_10(c, k, o)
    return tuple(int(v) for v in o)


def su3_field(n: int, eps: float, seed: int, tag: int = TAG_TRANSFORM, out: np.ndarray | None = None) -> np.ndarray:
    """``n`` SU(3) matrices ``exp(i eps H)`` as an ``(n, 3, 3)`` complex128 array."""
    if out is None:
        out = np.empty((n, 3, 3), dtype=np.complex128)
    _load().li_su3_field(_dptr(out.view(np.float64)), int(n), float(eps), int(seed), int(tag))
    return out


def gauge(dims, eps: float, seed: int, out: np.ndarray | None = None) -> np.ndarray:
    """Gauge field ``(V, 4, 3, 3)``; link (site, mu) keyed by index 4*site+mu."""
    v = volume(dims)
    if out is None:
        out = np.empty((v, 4, 3, 3), dtype=np.complex128)
    _load().li_su3_field(_dptr(out.view(np.float64)), 4 * v, float(eps), int(seed), TAG_GAUGE)
    return out


def unit_gauge(dims) -> np.ndarray:
    v = volume(dims)
    u = np.zeros((v, 4, 3, 3), dtype=np.complex128)
    u[:, :, 0, 0] = u[:, :, 1, 1] = u[:, :, 2, 2] = 1.0
    return u


def gaussian_spinor(dims, seed: int, out: np.ndarray | None = None) -> np.ndarray:
    """Complex-Gaussian spinor: re and im each N(0, 1)."""
    v = volume(dims)
    if out is None:
        out = np.empty((v, 4, 3), dtype=np.complex128)
    _load().li_gaussian(_dptr(out.view(np.float64)), 24 * v, int(seed), TAG_SPINOR)
    return out


def uniform_spinor(dims, seed: int) -> np.ndarray:
    """Spinor whose 24 real components per site are uniform in (0, 1)."""
    v = volume(dims)
    out = np.empty((v, 4, 3), dtype=np.complex128)
    _load().li_uniform(_dptr(out.view(np.float64)), 24 * v, int(seed), TAG_UNIFORM)
    return out


def point_source(dims, site=(0, 0, 0, 0), spin: int = 0, colour: int = 0) -> np.ndarray:
    x, y, z, t = site
    X, Y, Z, T = dims
    out = np.zeros((volume(dims), 4, 3), dtype=np.complex128)
    out[x + X * (y + Y * (z + Z * t)), spin, colour] = 1.0
    return out


def lex_index(dims, x, y, z, t):
    X, Y, Z, T = dims
    return x + X * (y + Y * (z + Z * t))


def coords(dims):
    """Integer coordinate arrays (x, y, z, t), each of length V, lexicographic order."""
    X, Y, Z, T = dims
    t, z, y, x = np.meshgrid(np.arange(T), np.arange(Z), np.arange(Y), np.arange(X), indexing="ij")
    return x.ravel(), y.ravel(), z.ravel(), t.ravel()


def parity(dims) -> np.ndarray:
    x, y, z, t = coords(dims)
    return (x + y + z + t) & 1
