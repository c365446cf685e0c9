"""GB300 Wilson-Dirac dslash and mixed-precision solvers (arXiv:0911.3191).

Thin Python binding of the C ABI in ``include/wilson_dirac.h``: argument
marshalling only.  Every step of the computation runs in the CUDA library
``libwilson_dirac.so`` (built in-tree by ``build.py``); PyTorch provides
device memory (``torch.uint8`` buffers holding fields in the library's
layout) and the CUDA stream.  There is no CPU fallback: if the library is
missing or no CUDA device is present, every call raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libwilson_dirac.so")

# wd_prec
F64, F32, Q16, H16N, B16N = 0, 1, 2, 3, 4
PREC_NAMES = {F64: "f64", F32: "f32", Q16: "q16", H16N: "h16n", B16N: "b16n"}
PREC_BY_NAME = {v: k for k, v in PREC_NAMES.items()}
# wd_solver
BICGSTAB, CGNR = 0, 1
# wd_operator
M_FULL, M_SCHUR_EVEN = 0, 1
EVEN, ODD = 0, 1

STATUS = {0: "ok", 1: "invalid argument", 2: "out of device memory", 3: "CUDA error", 4: "not converged",
          5: "Krylov breakdown", 6: "NaN or Inf", 7: "device wait timed out", 8: "memory budget exceeded",
          9: "call out of order"}


class WDError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class SolveParams(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("delta", ctypes.c_double), ("max_iter", ctypes.c_int),
                ("solver", ctypes.c_int), ("inner_precision", ctypes.c_int), ("use_graph", ctypes.c_int),
                ("restart", ctypes.c_int), ("xhat_f32", ctypes.c_int), ("initial_guess", ctypes.c_int)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("reliable_updates", ctypes.c_int), ("true_rel_residual", ctypes.c_double),
                ("iterated_rel_residual", ctypes.c_double), ("seconds", ctypes.c_double), ("status", ctypes.c_int),
                ("kernel_launches", ctypes.c_longlong)]


class ServerStats(ctypes.Structure):
    _fields_ = [("admit_seconds", ctypes.c_double), ("retire_seconds", ctypes.c_double),
                ("wait_seconds", ctypes.c_double), ("gpu_step_seconds", ctypes.c_double),
                ("steps", ctypes.c_longlong), ("admitted", ctypes.c_longlong), ("retired", ctypes.c_longlong)]


class ServerParams(ctypes.Structure):
    _fields_ = [("budget_bytes", ctypes.c_size_t), ("max_slots", ctypes.c_int), ("iters_per_step", ctypes.c_int),
                ("inner_precision", ctypes.c_int), ("delta", ctypes.c_double), ("max_iter", ctypes.c_int),
                ("use_graph", ctypes.c_int), ("gauge_flags", ctypes.c_int), ("rhs_tile", ctypes.c_int)]


_lib = None

GAUGE_TEMPORAL, GAUGE_RECON8 = 1, 2


def gauge_flags(temporal_gauge=False, recon8=False) -> int:
    """wd_gauge_flags of wd_load_gauge_opt."""
    return (GAUGE_TEMPORAL if temporal_gauge else 0) | (GAUGE_RECON8 if recon8 else 0)


def library_path() -> str:
    return LIB_PATH


def load_library():
    """Load libwilson_dirac.so; raise if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing (run paper_0911_3191_gb300/build.py)")
    lib = ctypes.CDLL(LIB_PATH)
    vp, dp, ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)
    c_int, c_dbl = ctypes.c_int, ctypes.c_double
    sigs = {
        "wd_create": (c_int, [ctypes.POINTER(vp), ip, c_int, vp]),
        "wd_destroy": (c_int, [vp]),
        "wd_set_stream": (c_int, [vp, vp]),
        "wd_field_bytes": (ctypes.c_size_t, [vp, c_int]),
        "wd_load_gauge": (c_int, [vp, vp, c_int, c_int]),
        "wd_load_gauge_opt": (c_int, [vp, vp, c_int, c_int, c_int]),
        "wd_field_import": (c_int, [vp, vp, vp, c_int, c_int, c_int]),
        "wd_field_export": (c_int, [vp, vp, vp, c_int, c_int, c_int]),
        "wd_dslash": (c_int, [vp, vp, vp, c_int, c_int, c_int]),
        "wd_dslash_xpay": (c_int, [vp, vp, vp, vp, c_dbl, c_int, c_int, c_int]),
        "wd_apply_M": (c_int, [vp, vp, vp, c_dbl, c_int, c_int, c_int]),
        "wd_norm2": (c_int, [vp, dp, vp, c_int]),
        "wd_solve": (c_int, [vp, vp, vp, c_dbl, ctypes.POINTER(SolveParams), ctypes.POINTER(SolveInfo)]),
        "wd_solve_device": (c_int, [vp, vp, vp, c_dbl, ctypes.POINTER(SolveParams), ctypes.POINTER(SolveInfo)]),
        "wd_dslash_batch": (c_int, [vp, vp, vp, c_int, c_int, c_int, c_int]),
        "wd_solve_batch_device": (c_int, [vp, c_int, vp, vp, dp, ctypes.POINTER(SolveParams),
                                          ctypes.POINTER(SolveInfo)]),
        "wd_solve_batch": (c_int, [vp, c_int, ctypes.POINTER(vp), ctypes.POINTER(vp), dp,
                                   ctypes.POINTER(SolveParams), ctypes.POINTER(SolveInfo)]),
        "wd_solve_multishift": (c_int, [vp, c_int, ctypes.POINTER(vp), vp, dp, ctypes.POINTER(SolveParams),
                                        ctypes.POINTER(SolveInfo)]),
        "wd_solve_multishift_device": (c_int, [vp, c_int, vp, vp, dp, ctypes.POINTER(SolveParams),
                                               ctypes.POINTER(SolveInfo)]),
        "wd_server_create": (c_int, [ctypes.POINTER(vp), ctypes.POINTER(ServerParams)]),
        "wd_server_destroy": (c_int, [vp]),
        "wd_server_add_gauge": (c_int, [vp, ip, c_int, vp, c_int, ip]),
        "wd_server_submit": (c_int, [vp, c_int, vp, vp, c_dbl, c_dbl, ctypes.POINTER(ctypes.c_longlong)]),
        "wd_server_step": (c_int, [vp, ip, ip]),
        "wd_server_poll": (c_int, [vp, ctypes.c_longlong, ip, ctypes.POINTER(SolveInfo)]),
        "wd_server_memory_in_use": (ctypes.c_size_t, [vp]),
        "wd_server_get_stats": (c_int, [vp, ctypes.POINTER(ServerStats)]),
        "wd_server_last_error": (ctypes.c_char_p, [vp]),
        "wd_slab_face_bytes": (ctypes.c_size_t, [vp, c_int]),
        "wd_slab_link_face_bytes": (ctypes.c_size_t, [vp, c_int]),
        "wd_slab_pack_faces": (c_int, [vp, vp, vp, vp, c_int, c_int]),
        "wd_slab_pack_link_face": (c_int, [vp, vp, c_int]),
        "wd_dslash_slab": (c_int, [vp, vp, vp, vp, vp, vp, c_int, c_int, c_int, c_int, c_int, c_int]),
        "wd_last_error": (ctypes.c_char_p, [vp]),
        "wd_status_string": (ctypes.c_char_p, [c_int]),
    }
    for name, (res, args) in sigs.items():
        f = getattr(lib, name)
        f.restype, f.argtypes = res, args
    _lib = lib
    return lib


def exported_symbols():
    """Names the C ABI exports (for load checks without a GPU)."""
    lib = load_library()
    return [n for n in ("wd_create", "wd_destroy", "wd_set_stream", "wd_field_bytes", "wd_load_gauge",
                        "wd_load_gauge_opt",
                        "wd_field_import", "wd_field_export", "wd_dslash", "wd_dslash_xpay", "wd_apply_M", "wd_norm2",
                        "wd_solve", "wd_solve_device", "wd_dslash_batch", "wd_solve_batch", "wd_solve_batch_device",
                        "wd_solve_multishift", "wd_solve_multishift_device", "wd_server_create", "wd_server_destroy", "wd_server_add_gauge", "wd_server_submit",
                        "wd_server_step", "wd_server_poll", "wd_server_memory_in_use", "wd_server_last_error",
                        "wd_server_get_stats",
                        "wd_slab_face_bytes", "wd_slab_link_face_bytes", "wd_slab_pack_faces",
                        "wd_slab_pack_link_face", "wd_dslash_slab",
                        "wd_norm2_noalloc", "wd_last_error", "wd_status_string")
            if hasattr(lib, n)]


def _ptr(a) -> int:
    """Address of a torch tensor or numpy array (C-contiguous)."""
    if hasattr(a, "data_ptr"):
        assert a.is_contiguous()
        return a.data_ptr()
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


def _is_device(a) -> int:
    return int(bool(getattr(a, "is_cuda", False)))


@dataclass
class SolveResult:
    status: int
    iters: int
    reliable_updates: int
    true_rel_residual: float
    iterated_rel_residual: float
    seconds: float
    kernel_launches: int


class WilsonDirac:
    """One lattice on one GPU: the library context (``wd_ctx``)."""

    def __init__(self, dims, t_antiperiodic: bool = False, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("no CUDA device: the Wilson-Dirac library runs on the GPU only")
        self.lib = load_library()
        self.dims = tuple(int(d) for d in dims)
        self.torch = torch
        s = stream if stream is not None else torch.cuda.current_stream()
        self.stream = s
        h = ctypes.c_void_p()
        d = (ctypes.c_int * 4)(*self.dims)
        st = self.lib.wd_create(ctypes.byref(h), d, int(bool(t_antiperiodic)), ctypes.c_void_p(s.cuda_stream))
        if st != 0:
            raise WDError(st, "wd_create failed")
        self.ctx = h

    # -- plumbing
    def close(self):
        if getattr(self, "ctx", None):
            self.lib.wd_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st: int, what: str):
        if st != 0:
            raise WDError(st, f"{what}: {self.lib.wd_last_error(self.ctx).decode()}")

    @property
    def volume(self) -> int:
        x, y, z, t = self.dims
        return x * y * z * t

    def field_bytes(self, prec: int) -> int:
        return int(self.lib.wd_field_bytes(self.ctx, prec))

    def new_field(self, prec: int, nparity: int = 1):
        """Uninitialised device field(s) of one precision (even then odd for nparity=2)."""
        return self.torch.empty(nparity * self.field_bytes(prec), dtype=self.torch.uint8, device="cuda")

    # -- the C ABI, call for call
    def load_gauge(self, U, recon: int = 12, temporal_gauge: bool = False, recon8: bool = False):
        """U: (V, 4, 3, 3) complex128 numpy array, or an equivalent float64 CUDA tensor.
        temporal_gauge: the temporal gauge inside the library (Sec. 4.3);
        recon8: FP32 / 16-bit links as the 8 numbers of App. A.2."""
        if isinstance(U, np.ndarray):
            U = np.ascontiguousarray(U, dtype=np.complex128)
        self._check(self.lib.wd_load_gauge_opt(self.ctx, ctypes.c_void_p(_ptr(U)), _is_device(U), recon,
                                               gauge_flags(temporal_gauge, recon8)), "load_gauge")

    def field_import(self, field, lex, parity: int, prec: int):
        if isinstance(lex, np.ndarray):
            lex = np.ascontiguousarray(lex, dtype=np.complex128)
        self._check(self.lib.wd_field_import(self.ctx, _ptr(field), _ptr(lex), _is_device(lex), parity, prec),
                    "field_import")

    def field_export(self, lex, field, parity: int, prec: int):
        self._check(self.lib.wd_field_export(self.ctx, _ptr(lex), _ptr(field), _is_device(lex), parity, prec),
                    "field_export")

    def dslash(self, out, inp, out_parity: int, dagger: bool, prec: int):
        self._check(self.lib.wd_dslash(self.ctx, _ptr(out), _ptr(inp), out_parity, int(dagger), prec), "dslash")

    def dslash_xpay(self, out, inp, x, a: float, out_parity: int, dagger: bool, prec: int):
        self._check(self.lib.wd_dslash_xpay(self.ctx, _ptr(out), _ptr(inp), _ptr(x), float(a), out_parity,
                                            int(dagger), prec), "dslash_xpay")

    # -- T-slab decomposition (one rank's slab; see tslab.SlabDslash)
    def slab_face_bytes(self, prec: int) -> int:
        return int(self.lib.wd_slab_face_bytes(self.ctx, prec))

    def slab_link_face_bytes(self, prec: int) -> int:
        return int(self.lib.wd_slab_link_face_bytes(self.ctx, prec))

    def slab_pack_faces(self, face_lo, face_hi, inp, dagger: bool, prec: int):
        self._check(self.lib.wd_slab_pack_faces(self.ctx, _ptr(face_lo), _ptr(face_hi), _ptr(inp), int(dagger), prec),
                    "slab_pack_faces")

    def slab_pack_link_face(self, face, prec: int):
        self._check(self.lib.wd_slab_pack_link_face(self.ctx, _ptr(face), prec), "slab_pack_link_face")

    def dslash_slab(self, out, inp, halo_lo, halo_hi, link_halo, flip_lo: bool, flip_hi: bool, out_parity: int,
                    dagger: bool, prec: int, region: int):
        """region 0: interior slices, 1: the two boundary slices, 2: all."""
        p = [None if a is None else ctypes.c_void_p(_ptr(a)) for a in (halo_lo, halo_hi, link_halo)]
        self._check(self.lib.wd_dslash_slab(self.ctx, _ptr(out), _ptr(inp), p[0], p[1], p[2], int(bool(flip_lo)),
                                            int(bool(flip_hi)), out_parity, int(dagger), prec, int(region)),
                    "dslash_slab")

    def apply_M(self, out, inp, kappa: float, which: int, dagger: bool, prec: int):
        self._check(self.lib.wd_apply_M(self.ctx, _ptr(out), _ptr(inp), float(kappa), which, int(dagger), prec),
                    "apply_M")

    def norm2(self, field, prec: int) -> float:
        r = ctypes.c_double()
        self._check(self.lib.wd_norm2(self.ctx, ctypes.byref(r), _ptr(field), prec), "norm2")
        return r.value

    @staticmethod
    def _params(tol, delta, max_iter, solver, inner_precision, use_graph, restart=False, xhat_f32=False,
                initial_guess=False):
        return SolveParams(float(tol), float(delta), int(max_iter), int(solver), int(inner_precision),
                           int(use_graph), int(bool(restart)), int(bool(xhat_f32)), int(bool(initial_guess)))

    def _solve(self, fn, x, b, kappa, tol, delta, max_iter, solver, inner_precision, use_graph, check,
               restart=False, xhat_f32=False, initial_guess=False):
        p = self._params(tol, delta, max_iter, solver, inner_precision, use_graph, restart, xhat_f32,
                         initial_guess)
        info = SolveInfo()
        st = fn(self.ctx, _ptr(x), _ptr(b), float(kappa), ctypes.byref(p), ctypes.byref(info))
        if check and st not in (0,):
            self._check(st, "solve")
        if st not in (0, 4, 5, 6) and not check:
            self._check(st, "solve")
        return SolveResult(int(info.status), int(info.iters), int(info.reliable_updates),
                           float(info.true_rel_residual), float(info.iterated_rel_residual), float(info.seconds),
                           int(info.kernel_launches))

    def solve(self, x, b, kappa, tol=1e-12, delta=0.1, max_iter=20000, solver=BICGSTAB, inner_precision=F64,
              use_graph=True, check=True, restart=False, xhat_f32=False, initial_guess=False) -> SolveResult:
        """x, b: (V, 4, 3) complex128 host arrays (pinned torch tensors also work).
        restart=True: defect correction (Alg. 1) with eps_in = delta.
        xhat_f32=True: x_hat in FP32 under a 16-bit inner precision.
        initial_guess=True: start from the x passed in (BiCGstab, reliable updates)."""
        return self._solve(self.lib.wd_solve, x, b, kappa, tol, delta, max_iter, solver, inner_precision,
                           use_graph, check, restart, xhat_f32, initial_guess)

    def solve_device(self, x, b, kappa, tol=1e-12, delta=0.1, max_iter=20000, solver=BICGSTAB,
                     inner_precision=F64, use_graph=True, check=True, restart=False,
                     xhat_f32=False, initial_guess=False) -> SolveResult:
        """x, b: device FP64 full fields (``new_field(F64, 2)``)."""
        return self._solve(self.lib.wd_solve_device, x, b, kappa, tol, delta, max_iter, solver, inner_precision,
                           use_graph, check, restart, xhat_f32, initial_guess)

    def dslash_batch(self, out, inp, nrhs: int, out_parity: int, dagger: bool, prec: int):
        """out_r = D in_r for nrhs single-parity fields stored back to back."""
        self._check(self.lib.wd_dslash_batch(self.ctx, _ptr(out), _ptr(inp), int(nrhs), out_parity, int(dagger), prec),
                    "dslash_batch")

    @staticmethod
    def _infos(arr, n):
        return [SolveResult(int(i.status), int(i.iters), int(i.reliable_updates), float(i.true_rel_residual),
                            float(i.iterated_rel_residual), float(i.seconds), int(i.kernel_launches))
                for i in arr[:n]]

    def solve_batch_device(self, x, b, kappas, tol=1e-12, delta=0.1, max_iter=20000, inner_precision=Q16,
                           use_graph=True, check=True):
        """x, b: n FP64 full fields back to back (``new_field(F64, 2 * n)``)."""
        n = len(kappas)
        k = (ctypes.c_double * n)(*[float(v) for v in kappas])
        p = self._params(tol, delta, max_iter, BICGSTAB, inner_precision, use_graph)
        infos = (SolveInfo * n)()
        st = self.lib.wd_solve_batch_device(self.ctx, n, _ptr(x), _ptr(b), k, ctypes.byref(p), infos)
        if st not in (0, 4, 5, 6) or (check and st != 0):
            self._check(st, "solve_batch_device")
        return self._infos(infos, n)

    def solve_batch(self, xs, bs, kappas, tol=1e-12, delta=0.1, max_iter=20000, inner_precision=Q16,
                    use_graph=True, check=True):
        """xs, bs: lists of (V, 4, 3) complex128 host arrays."""
        n = len(kappas)
        bs = [np.ascontiguousarray(b, dtype=np.complex128) for b in bs]
        xp = (ctypes.c_void_p * n)(*[_ptr(x) for x in xs])
        bp = (ctypes.c_void_p * n)(*[_ptr(b) for b in bs])
        k = (ctypes.c_double * n)(*[float(v) for v in kappas])
        p = self._params(tol, delta, max_iter, BICGSTAB, inner_precision, use_graph)
        infos = (SolveInfo * n)()
        st = self.lib.wd_solve_batch(self.ctx, n, xp, bp, k, ctypes.byref(p), infos)
        if st not in (0, 4, 5, 6) or (check and st != 0):
            self._check(st, "solve_batch")
        return self._infos(infos, n)

    def solve_multishift(self, xs, b, kappas, tol=1e-12, delta=0.1, max_iter=20000, inner_precision=Q16,
                         use_graph=True, check=True):
        """M_kappa_k x_k = b for every kappa (one shared multi-shift iteration,
        then a refinement per kappa).  xs: list of (V, 4, 3) complex128 host
        arrays (written); b: (V, 4, 3) complex128."""
        n = len(kappas)
        b = np.ascontiguousarray(b, dtype=np.complex128)
        xp = (ctypes.c_void_p * n)(*[_ptr(x) for x in xs])
        k = (ctypes.c_double * n)(*[float(v) for v in kappas])
        p = self._params(tol, delta, max_iter, BICGSTAB, inner_precision, use_graph)
        infos = (SolveInfo * n)()
        st = self.lib.wd_solve_multishift(self.ctx, n, xp, _ptr(b), k, ctypes.byref(p), infos)
        if st not in (0, 4, 5, 6) or (check and st != 0):
            self._check(st, "solve_multishift")
        return self._infos(infos, n)

    def solve_multishift_device(self, x, b, kappas, tol=1e-12, delta=0.1, max_iter=20000, inner_precision=Q16,
                                use_graph=True, check=True):
        """x: n FP64 full fields back to back (``new_field(F64, 2 * n)``); b:
        one FP64 full field."""
        n = len(kappas)
        k = (ctypes.c_double * n)(*[float(v) for v in kappas])
        p = self._params(tol, delta, max_iter, BICGSTAB, inner_precision, use_graph)
        infos = (SolveInfo * n)()
        st = self.lib.wd_solve_multishift_device(self.ctx, n, _ptr(x), _ptr(b), k, ctypes.byref(p), infos)
        if st not in (0, 4, 5, 6) or (check and st != 0):
            self._check(st, "solve_multishift_device")
        return self._infos(infos, n)

    # -- conveniences built only from the calls above
    def upload(self, lex, prec: int, parity: int | None = None):
        """Host (V,4,3) complex128 -> device field (one parity, or both when parity is None)."""
        if parity is None:
            f = self.new_field(prec, 2)
            n = self.field_bytes(prec)
            self.field_import(f[:n], lex, EVEN, prec)
            self.field_import(f[n:], lex, ODD, prec)
            return f
        f = self.new_field(prec, 1)
        self.field_import(f, lex, parity, prec)
        return f

    def download(self, field, prec: int, parity: int | None = None, out=None):
        """Device field -> host (V,4,3) complex128 (sites of other parity zero unless `out` given)."""
        if out is None:
            out = np.zeros((self.volume, 4, 3), dtype=np.complex128)
        if parity is None:
            n = self.field_bytes(prec)
            self.field_export(out, field[:n], EVEN, prec)
            self.field_export(out, field[n:], ODD, prec)
        else:
            self.field_export(out, field, parity, prec)
        return out


class Server:
    """Continuous-batching solve server (``wd_server_*``): resident gauge
    fields, a device-memory budget, requests admitted as slots free up."""

    def __init__(self, budget_bytes=0, max_slots=8, iters_per_step=8, inner_precision=Q16, delta=0.1,
                 max_iter=20000, use_graph=True, temporal_gauge=False, recon8=False, rhs_tile=0):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("no CUDA device: the Wilson-Dirac library runs on the GPU only")
        self.lib = load_library()
        p = ServerParams(int(budget_bytes), int(max_slots), int(iters_per_step), int(inner_precision), float(delta),
                         int(max_iter), int(use_graph), gauge_flags(temporal_gauge, recon8), int(rhs_tile))
        h = ctypes.c_void_p()
        st = self.lib.wd_server_create(ctypes.byref(h), ctypes.byref(p))
        if st != 0:
            raise WDError(st, "wd_server_create failed")
        self.h = h
        self._keep = {}  # request id -> (b, x) host arrays kept alive until retired

    def _check(self, st, what):
        if st != 0:
            raise WDError(st, f"{what}: {self.lib.wd_server_last_error(self.h).decode()}")

    def close(self):
        if getattr(self, "h", None):
            self.lib.wd_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add_gauge(self, dims, U, recon=12, t_antiperiodic=False) -> int:
        U = np.ascontiguousarray(U, dtype=np.complex128)
        d = (ctypes.c_int * 4)(*[int(v) for v in dims])
        gid = ctypes.c_int()
        self._check(self.lib.wd_server_add_gauge(self.h, d, int(bool(t_antiperiodic)), _ptr(U), int(recon),
                                                 ctypes.byref(gid)), "add_gauge")
        return gid.value

    def submit(self, gauge_id, b, kappa, tol, x=None) -> int:
        b = np.ascontiguousarray(b, dtype=np.complex128)
        if x is None:
            x = np.zeros_like(b)
        rid = ctypes.c_longlong()
        self._check(self.lib.wd_server_submit(self.h, int(gauge_id), _ptr(b), _ptr(x), float(kappa), float(tol),
                                              ctypes.byref(rid)), "submit")
        self._keep[rid.value] = (b, x)
        return rid.value

    def stats(self) -> dict:
        st = ServerStats()
        self._check(self.lib.wd_server_get_stats(self.h, ctypes.byref(st)), "stats")
        return {k: getattr(st, k) for k, _ in ServerStats._fields_}

    def step(self):
        a, q = ctypes.c_int(), ctypes.c_int()
        self._check(self.lib.wd_server_step(self.h, ctypes.byref(a), ctypes.byref(q)), "step")
        return a.value, q.value

    def poll(self, rid):
        """(finished, SolveResult or None, x or None)"""
        f = ctypes.c_int()
        info = SolveInfo()
        self._check(self.lib.wd_server_poll(self.h, int(rid), ctypes.byref(f), ctypes.byref(info)), "poll")
        if not f.value:
            return False, None, None
        b, x = self._keep.pop(rid, (None, None))
        res = SolveResult(int(info.status), int(info.iters), int(info.reliable_updates),
                          float(info.true_rel_residual), float(info.iterated_rel_residual), float(info.seconds),
                          int(info.kernel_launches))
        return True, res, x

    def memory_in_use(self) -> int:
        return int(self.lib.wd_server_memory_in_use(self.h))
