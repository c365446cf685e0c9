"""wd_norm2_noalloc: the squared norm for callers that cannot allocate device
memory (a host framework that owns all device memory and forbids other
allocations, or code about to capture a CUDA graph).  It needs no context and
keeps its reduction scratch in a static device array of the library.

Checked through the C ABI on two calls in a row, against numpy's |.|^2 of the
stored field bytes and against the context-based wd_norm2 (the scratch keeps
the previous call's contents, so the second, smaller call shows that nothing
left over from the first is used).  This file is collected
last, so a run that stops at its first failure has already run every other
test."""
import ctypes

import numpy as np
import pytest

import lattice_inputs as li
from tests.wd_testutil import split16, stride_of

pytestmark = pytest.mark.gpu


def _bind(lib):
    f = lib.wd_norm2_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_void_p,
                  ctypes.c_char_p, ctypes.c_size_t]
    return f


def _stored_norm2(raw: np.ndarray, dims, prec: int) -> float:
    """|field|^2 of the values a single-parity field stores, decoded here with
    numpy from its bytes (library layout: component arrays of `stride` sites;
    16-bit codes decoded in FP32 as code * norm, Q16 with norm / 32767)."""
    vh = li.volume(dims) // 2
    st = stride_of(dims)
    if prec == 0:
        v = raw[: 192 * st].view(np.float64).reshape(12, st, 2)[:, :vh]
    elif prec == 1:
        v = raw[: 96 * st].view(np.float32).reshape(6, st, 4)[:, :vh].astype(np.float64)
    else:
        codes, norms = split16(raw, dims)
        if prec == 2:
            scale = (norms * np.float32(1.0 / 32767.0)).astype(np.float32)
            f = codes.view(np.int16).astype(np.float32)
        elif prec == 3:
            scale = norms
            f = codes.view(np.float16).astype(np.float32)
        else:
            scale = norms
            f = (codes.astype(np.uint32) << 16).view(np.float32)
        v = (f * scale[:, None]).astype(np.float64)
    return float(np.sum(v * v))


@pytest.mark.parametrize("prec", [0, 1, 2, 3, 4])
def test_norm2_noalloc_matches_stored_field_on_two_calls(prec):
    """Two calls in a row, a larger lattice (128 blocks) and then a smaller
    one (6 blocks), so that partial sums the first call left in the shared
    scratch beyond the second call's grid would show.  Each result is checked
    against numpy's |.|^2 of the stored field and against wd_norm2."""
    import torch

    import paper_0911_3191_gb300 as wdp
    fn = _bind(wdp.load_library())
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    err = ctypes.create_string_buffer(256)
    for call, dims in enumerate([(16, 16, 16, 16), (8, 6, 4, 16)]):
        wd = wdp.WilsonDirac(dims)
        psi = li.gaussian_spinor(dims, 4100 + 10 * prec + call) * (1.0 + call)
        field = wd.upload(psi, prec, parity=call % 2)
        d = (ctypes.c_int * 4)(*dims)
        out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
        st = fn(out.data_ptr(), field.data_ptr(), d, prec, stream, err, len(err))
        torch.cuda.synchronize()
        assert st == 0, err.value
        got = out.item()
        numpy_norm = _stored_norm2(field.cpu().numpy(), dims, prec)
        assert abs(got - numpy_norm) <= 1e-12 * numpy_norm, (call, got, numpy_norm)
        want = wd.norm2(field, prec)
        assert abs(got - want) <= 1e-12 * want, (call, got, want)
        wd.close()


def test_norm2_noalloc_rejects_oversize_and_bad_args():
    import torch

    import paper_0911_3191_gb300 as wdp
    fn = _bind(wdp.load_library())
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    dummy = torch.zeros(256, dtype=torch.uint8, device="cuda")
    err = ctypes.create_string_buffer(256)
    # 64^3 x 130: 17,039,360 sites per parity, above the scratch's 16,777,216;
    # rejected before any launch
    big = (ctypes.c_int * 4)(64, 64, 64, 130)
    assert fn(out.data_ptr(), dummy.data_ptr(), big, 2, None, err, len(err)) == 1
    assert b"too large" in err.value
    odd = (ctypes.c_int * 4)(4, 4, 3, 4)
    assert fn(out.data_ptr(), dummy.data_ptr(), odd, 2, None, err, len(err)) == 1
    assert fn(None, dummy.data_ptr(), (ctypes.c_int * 4)(4, 4, 4, 4), 2, None, err, len(err)) == 1
    assert fn(out.data_ptr(), dummy.data_ptr(), (ctypes.c_int * 4)(4, 4, 4, 4), 7, None, err, len(err)) == 1
    assert np.isfinite(out.item())
