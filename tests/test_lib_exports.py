"""CPU-side checks of the C-ABI library: it loads and exports every symbol include/polfed.h declares."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "polfed.h")


def _declared():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = set(re.findall(r"\b(pf_[A-Za-z0-9_]+)\s*\(", txt))
    return {n for n in names if not n.endswith("_fn")}


@pytest.fixture(scope="module")
def libpath():
    from paper_2605_10191_b300 import build as b
    return b.build()


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_prototypes_cover_header(libpath):
    from paper_2605_10191_b300 import _lib
    assert _declared() == set(_lib.PROTOTYPES)


def test_status_strings_without_gpu(libpath):
    from paper_2605_10191_b300 import _lib
    L = _lib.lib()
    assert L.pf_status_str(0) == b"PF_OK"
    assert b"PF_EINVAL" in L.pf_status_str(1)
    o = _lib.pf_solve_opts()
    L.pf_default_opts(ctypes.byref(o))
    assert o.block == 32 and abs(o.tol - 1e-10) < 1e-25 and abs(o.res_tol - 1e-9) < 1e-24


def test_invalid_arguments_rejected_without_gpu(libpath):
    from paper_2605_10191_b300 import _lib
    L = _lib.lib()
    # NULL model / NULL handle are rejected before any CUDA call
    h = ctypes.c_void_p()
    assert L.pf_build_basis(None, ctypes.byref(h), None) == _lib.PF_EINVAL
    assert L.pf_polfed_solve(None, 0.5, 1, 10, None, None, None, None, None, None) == _lib.PF_EINVAL
    assert L.pf_filter_coefficients(2.0, 10, None, None) == _lib.PF_EINVAL
