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


def _c_layout(structs, constants, tmp_path):
    """sizeof/offsetof of the header's structs and the values of its constants, from a C program
    compiled against include/polfed.h with the host compiler."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ["#include <stdio.h>", "#include <stddef.h>", f'#include "{HEADER}"', "int main(void) {"]
    for name, fields in structs.items():
        lines.append(f'  printf("{name} %zu\\n", sizeof({name}));')
        for f in fields:
            cf = f[:-1] if f.endswith("_") else f      # Python names avoid keywords (lambda_)
            lines.append(f'  printf("{name}.{f} %zu\\n", offsetof({name}, {cf}));')
    for c in constants:
        lines.append(f'  printf("{c} %ld\\n", (long){c});')
    lines.append("  return 0;\n}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-o", str(exe), str(src)], check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    return dict((k, int(v)) for k, v in (l.split() for l in out.strip().splitlines()))


def test_binding_structs_and_constants_match_header(tmp_path):
    """Every ctypes structure of the binding has the C layout (size, field offsets) and every
    constant the header's value: a field added on one side only shows up here, without a GPU."""
    from paper_2605_10191_b300 import _lib
    structs = {n: [f[0] for f in getattr(_lib, n)._fields_]
               for n in ("pf_model", "pf_params", "pf_solve_opts", "pf_report", "pf_filter_item", "pf_solve_item",
                         "pf_server_config", "pf_request_info")}
    consts = ["PF_OK", "PF_EINVAL", "PF_ENOMEM", "PF_ENOTCONV", "PF_ETIMEOUT", "PF_ECUDA", "PF_ESTATE",
              "PF_EBREAKDOWN", "PF_MODEL_XXZ", "PF_MODEL_QSUN", "PF_MODEL_HUBBARD", "PF_MODEL_QREM",
              "PF_MODEL_QSUN_U1", "PF_MAP_CSR", "PF_MAP_STRUCTURED", "PF_F64", "PF_F32", "PF_DF64",
              "PF_FORM_AUTO", "PF_FORM_STEPS", "PF_FORM_GRAPH", "PF_REFINE_DIRECT", "PF_REFINE_CORRECTION"]
    got = _c_layout(structs, consts, tmp_path)
    for n, fields in structs.items():
        cls = getattr(_lib, n)
        assert ctypes.sizeof(cls) == got[n], n
        for f in fields:
            assert getattr(cls, f).offset == got[f"{n}.{f}"], (n, f)
    for c in consts:
        assert getattr(_lib, c) == got[c], c
