"""wd_norm2_noalloc: the squared norm for callers that cannot allocate device
memory (a host framework that owns all device memory and forbids other
allocations, or code about to capture a CUDA graph).  It needs no context and
keeps its reduction scratch in a static device array of the library.

Checked through the C ABI against the context-based wd_norm2 on the same
fields, on two calls in a row (the scratch keeps the previous call's contents,
so the second call shows it is cleared correctly).  This file is collected
last, so a run that stops at its first failure has already run every other
test."""
import ctypes

import numpy as np
import pytest

import lattice_inputs as li

pytestmark = pytest.mark.gpu


def _bind(lib):
    f = lib.wd_norm2_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_void_p,
                  ctypes.c_char_p, ctypes.c_size_t]
    return f


@pytest.mark.parametrize("prec", [0, 1, 2, 3, 4])
def test_norm2_noalloc_matches_norm2_on_two_calls(prec):
    import torch

    import paper_0911_3191_gb300 as wdp
    lib = wdp.load_library()
    fn = _bind(lib)
    dims = (8, 6, 4, 16)
    wd = wdp.WilsonDirac(dims)
    psi = li.gaussian_spinor(dims, 4100 + prec)
    d = (ctypes.c_int * 4)(*dims)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    err = ctypes.create_string_buffer(256)
    for call in range(2):
        field = wd.upload(psi * (1.0 + call), prec, parity=call % 2)
        want = wd.norm2(field, prec)
        out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
        st = fn(out.data_ptr(), field.data_ptr(), d, prec, stream, err, len(err))
        torch.cuda.synchronize()
        assert st == 0, err.value
        got = out.item()
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
