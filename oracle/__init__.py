"""ORACLE -- test infrastructure only.

Python access to the plain FP64 CPU Wilson-Dirac implementation in
``wd_oracle.c`` (operator, Schur complement, BiCGstab, CG on the normal
equations, 16-bit storage codecs).  Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` use it; the CUDA library and its
Python binding never import it, and nothing here imports them.

Conventions (arXiv:0911.3191, Sec. 3 and App. B): fields are full-lattice,
lexicographic, DeGrand-Rossi basis, numpy complex128:

* spinor ``(V, 4, 3)``, gauge ``(V, 4, 3, 3)``; site ``x + X(y + Y(z + Z t))``
* ``M_kappa = 1 - kappa D``; ``M_hat = 1 - kappa^2 D_eo D_oe`` on even sites

Parity status of every function: pinned (see ``tests/test_oracle_pins.py``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wd_oracle.c")
_LIB = os.path.join(_HERE, "_wd_oracle.so")
_lock = threading.Lock()
_lib = None

FMT_Q16, FMT_H16N, FMT_B16N = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle (gcc, FP64, OpenMP, no floating-point contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                               "-fcx-limited-range", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int)
            i64p = ctypes.POINTER(ctypes.c_int64)
            i16p = ctypes.POINTER(ctypes.c_int16)
            fp = ctypes.POINTER(ctypes.c_float)
            c_int, c_dbl, c_i64 = ctypes.c_int, ctypes.c_double, ctypes.c_int64
            sig = {
                "wo_gamma": (None, [c_int, dp]),
                "wo_dslash": (None, [dp, dp, dp, ip, c_int, c_int, c_int]),
                "wo_dslash_sites": (None, [dp, dp, dp, ip, c_int, c_int, i64p, c_i64]),
                "wo_apply_M": (None, [dp, dp, dp, ip, c_int, c_dbl, c_int]),
                "wo_apply_Mhat": (None, [dp, dp, dp, ip, c_int, c_dbl, c_int]),
                "wo_solve": (c_int, [dp, dp, dp, ip, c_int, c_dbl, c_dbl, c_int, c_int, c_int, dp]),
                "wo_bicgstab_schur_iters": (c_dbl, [dp, dp, ip, c_int, c_dbl, c_int]),
                "wo_encode_spinor": (None, [dp, c_i64, c_int, i16p, fp, fp]),
                "wo_decode_spinor": (None, [i16p, fp, fp, c_i64, c_int, dp]),
                "wo_encode_link_values": (None, [dp, c_i64, c_int, i16p, dp]),
                "wo_su3_to8": (c_int, [dp, dp]),
                "wo_su3_from8": (None, [dp, dp]),
                "wo_round_fp16": (ctypes.c_float, [ctypes.c_float]),
                "wo_round_bf16": (ctypes.c_float, [ctypes.c_float]),
            }
            for name, (res, args) in sig.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def _p(a: np.ndarray, ctype=ctypes.c_double):
    assert a.flags["C_CONTIGUOUS"], "oracle arrays must be C-contiguous"
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _dims(dims):
    d = (ctypes.c_int * 4)(*[int(v) for v in dims])
    return d


def _f64(a: np.ndarray) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.complex128)
    return a.view(np.float64)


def gamma(mu: int) -> np.ndarray:
    """gamma_mu (mu = 0..3 <-> x, y, z, t), DeGrand-Rossi basis, 4x4 complex."""
    out = np.zeros((4, 4), dtype=np.complex128)
    _load().wo_gamma(int(mu), _p(out.view(np.float64)))
    return out


def dslash(psi, U, dims, dagger=False, out_parity=-1, tbc_anti=False) -> np.ndarray:
    """D psi (or D^dag psi); ``out_parity`` 0/1 keeps only that parity's sites."""
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    U = np.ascontiguousarray(U, dtype=np.complex128)
    out = np.empty_like(psi)
    _load().wo_dslash(_p(out.view(np.float64)), _p(psi.view(np.float64)), _p(U.view(np.float64)),
                      _dims(dims), int(tbc_anti), int(dagger), int(out_parity))
    return out


def dslash_sites(psi, U, dims, sites, dagger=False, tbc_anti=False) -> np.ndarray:
    """D psi at the listed lexicographic sites only: ``(n, 4, 3)``."""
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    U = np.ascontiguousarray(U, dtype=np.complex128)
    sites = np.ascontiguousarray(sites, dtype=np.int64)
    out = np.empty((len(sites), 4, 3), dtype=np.complex128)
    _load().wo_dslash_sites(_p(out.view(np.float64)), _p(psi.view(np.float64)), _p(U.view(np.float64)),
                            _dims(dims), int(tbc_anti), int(dagger), _p(sites, ctypes.c_int64), len(sites))
    return out


def apply_M(psi, U, dims, kappa, dagger=False, tbc_anti=False) -> np.ndarray:
    """M_kappa psi = psi - kappa D psi (full lattice)."""
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    U = np.ascontiguousarray(U, dtype=np.complex128)
    out = np.empty_like(psi)
    _load().wo_apply_M(_p(out.view(np.float64)), _p(psi.view(np.float64)), _p(U.view(np.float64)),
                       _dims(dims), int(tbc_anti), float(kappa), int(dagger))
    return out


def apply_Mhat(psi, U, dims, kappa, dagger=False, tbc_anti=False) -> np.ndarray:
    """(1 - kappa^2 D_eo D_oe) psi_e on even sites; odd sites of the result are 0."""
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    U = np.ascontiguousarray(U, dtype=np.complex128)
    out = np.empty_like(psi)
    _load().wo_apply_Mhat(_p(out.view(np.float64)), _p(psi.view(np.float64)), _p(U.view(np.float64)),
                          _dims(dims), int(tbc_anti), float(kappa), int(dagger))
    return out


def solve(b, U, dims, kappa, tol=1e-12, maxiter=10000, solver="bicgstab", schur=True, tbc_anti=False):
    """FP64 solve of M_kappa x = b.  Returns (x, status, iterations, true |b-Mx|/|b|)."""
    b = np.ascontiguousarray(b, dtype=np.complex128)
    U = np.ascontiguousarray(U, dtype=np.complex128)
    x = np.empty_like(b)
    info = np.zeros(2, dtype=np.float64)
    s = {"bicgstab": 0, "cgnr": 1}[solver]
    st = _load().wo_solve(_p(x.view(np.float64)), _p(b.view(np.float64)), _p(U.view(np.float64)), _dims(dims),
                          int(tbc_anti), float(kappa), float(tol), int(maxiter), s, int(bool(schur)),
                          _p(info))
    return x, int(st), int(info[0]), float(info[1])


def bicgstab_schur_iterations(b, U, dims, kappa, iterations, tbc_anti=False) -> float:
    """Run exactly ``iterations`` Schur BiCGstab iterations (a bounded timing sample)."""
    b = np.ascontiguousarray(b, dtype=np.complex128)
    U = np.ascontiguousarray(U, dtype=np.complex128)
    return float(_load().wo_bicgstab_schur_iters(_p(b.view(np.float64)), _p(U.view(np.float64)), _dims(dims),
                                                  int(tbc_anti), float(kappa), int(iterations)))


def true_residual(x, b, U, dims, kappa, tbc_anti=False) -> float:
    """|b - M_kappa x| / |b| in FP64."""
    r = np.asarray(b) - apply_M(x, U, dims, kappa, tbc_anti=tbc_anti)
    return float(np.linalg.norm(r) / np.linalg.norm(b))


def encode_spinor(v, fmt: int):
    """Per-site 16-bit codec (Sec. 4.6).  ``v``: (n, 24) or (n, 4, 3) complex.

    Returns (codes int16 (n, 24) for Q16 else None, rounded values float32
    (n, 24) for H16N/B16N else None, norms float32 (n,))."""
    v = np.ascontiguousarray(np.asarray(v, dtype=np.complex128)).reshape(-1, 12).view(np.float64)
    v = np.ascontiguousarray(v)
    n = v.shape[0]
    codes = np.zeros((n, 24), dtype=np.int16)
    vals = np.zeros((n, 24), dtype=np.float32)
    norms = np.zeros(n, dtype=np.float32)
    _load().wo_encode_spinor(_p(v), n, int(fmt), _p(codes, ctypes.c_int16), _p(vals, ctypes.c_float),
                             _p(norms, ctypes.c_float))
    return (codes if fmt == FMT_Q16 else None), (vals if fmt != FMT_Q16 else None), norms


def decode_spinor(codes, vals, norms, fmt: int) -> np.ndarray:
    """Decoded float values (as float64) ``(n, 24)``."""
    n = len(norms)
    codes = np.ascontiguousarray(codes if codes is not None else np.zeros((n, 24), np.int16), dtype=np.int16)
    vals = np.ascontiguousarray(vals if vals is not None else np.zeros((n, 24), np.float32), dtype=np.float32)
    norms = np.ascontiguousarray(norms, dtype=np.float32)
    out = np.zeros((n, 24), dtype=np.float64)
    _load().wo_decode_spinor(_p(codes, ctypes.c_int16), _p(vals, ctypes.c_float), _p(norms, ctypes.c_float), n,
                             int(fmt), _p(out))
    return out


def quantise_spinor(v, fmt: int) -> np.ndarray:
    """Round trip through a 16-bit format: the values a kernel sees. Same shape as v."""
    shape = np.shape(v)
    c, w, nrm = encode_spinor(v, fmt)
    d = decode_spinor(c, w, nrm, fmt)
    return d.view(np.complex128).reshape(shape)


def encode_link_values(u, fmt: int):
    """16-bit link storage of real values ``u`` (flat float64).  Returns (codes, decoded)."""
    u = np.ascontiguousarray(u, dtype=np.float64).ravel()
    codes = np.zeros(u.shape, dtype=np.int16)
    dec = np.zeros(u.shape, dtype=np.float64)
    _load().wo_encode_link_values(_p(u), len(u), int(fmt), _p(codes, ctypes.c_int16), _p(dec))
    return codes, dec


def quantise_gauge(U, fmt: int) -> np.ndarray:
    """The gauge field as a 16-bit-link kernel sees it (all 18 reals rounded)."""
    U = np.ascontiguousarray(U, dtype=np.complex128)
    _, dec = encode_link_values(U.view(np.float64), fmt)
    return dec.view(np.complex128).reshape(U.shape)


def round_fp16(w: float) -> float:
    return float(_load().wo_round_fp16(float(w)))


def round_bf16(w: float) -> float:
    return float(_load().wo_round_bf16(float(w)))


def su3_to8(U) -> tuple:
    """App. A.2: links (..., 3, 3) -> (p (..., 8), singular (...,) bool)."""
    U = np.ascontiguousarray(U, dtype=np.complex128)
    flat = U.reshape(-1, 9)
    p = np.empty((len(flat), 8), dtype=np.float64)
    sing = np.empty(len(flat), dtype=bool)
    lib = _load()
    for i in range(len(flat)):
        row = np.ascontiguousarray(flat[i])
        out = np.empty(8)
        sing[i] = bool(lib.wo_su3_to8(_p(row.view(np.float64)), _p(out)))
        p[i] = out
    return p.reshape(U.shape[:-2] + (8,)), sing.reshape(U.shape[:-2])


def su3_from8(p) -> np.ndarray:
    """App. A.2: (..., 8) parameters -> links (..., 3, 3)."""
    p = np.ascontiguousarray(p, dtype=np.float64)
    flat = p.reshape(-1, 8)
    out = np.empty((len(flat), 9), dtype=np.complex128)
    lib = _load()
    for i in range(len(flat)):
        row = np.ascontiguousarray(flat[i])
        o = np.empty(9, dtype=np.complex128)
        lib.wo_su3_from8(_p(row), _p(o.view(np.float64)))
        out[i] = o
    return out.reshape(p.shape[:-1] + (3, 3))
