"""The C-ABI library builds, loads without a GPU, and exports every entry
point that include/wilson_dirac.h declares.  No compute call is made here."""
import os
import re
import subprocess

import pytest

import paper_0911_3191_gb300 as wdp
from paper_0911_3191_gb300 import build as cuda_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"^\s*(?:const\s+)?[\w]+\s*\*?\s*(wd_\w+)\s*\(", src, flags=re.M))
    return sorted(names)


@pytest.fixture(scope="module")
def lib_path():
    return cuda_build.build()


def test_header_declares_the_boundary():
    names = declared_entry_points()
    for n in ("wd_create", "wd_load_gauge", "wd_dslash", "wd_apply_M", "wd_solve", "wd_field_import"):
        assert n in names


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s+(wd_\w+)$", out, flags=re.M))
    missing = [n for n in declared_entry_points() if n not in exported]
    assert not missing, f"declared but not exported: {missing}"


def test_library_loads_and_binds_without_gpu(lib_path):
    lib = wdp.load_library()
    assert set(declared_entry_points()) <= set(wdp.exported_symbols())
    assert lib.wd_status_string(4) == b"not converged"
    assert lib.wd_last_error(None) == b"null context"


def test_bad_dims_rejected_without_touching_a_gpu(lib_path):
    import ctypes
    lib = wdp.load_library()
    h = ctypes.c_void_p()
    for dims in ((3, 4, 4, 4), (4, 4, 4, 0), (4, 4, -2, 4)):
        d = (ctypes.c_int * 4)(*dims)
        assert lib.wd_create(ctypes.byref(h), d, 0, None) == 1  # WD_ERR_INVALID_ARG


def test_no_oracle_in_the_product_path():
    """The package and its sources never import or link the oracle."""
    pkg = os.path.join(ROOT, "paper_0911_3191_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in src and "from oracle" not in src and "wd_oracle" not in src, f
