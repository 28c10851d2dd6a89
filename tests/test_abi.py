"""The C-ABI library builds, loads and exports every function include/gw.h
declares.  No compute call is made (runs without a GPU)."""
import ctypes
import os

import pytest

from paper_2404_08970_gb300 import _lib as L


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(L.LIB_PATH):
        from paper_2404_08970_gb300 import build
        build.build()
    return L.load()


def test_exports_every_declared_symbol(lib):
    names = L.declared_functions()
    assert "gw_grad" in names
    raw = ctypes.CDLL(L.LIB_PATH)
    missing = [n for n in names if not hasattr(raw, n)]
    assert not missing, f"declared but not exported: {missing}"


def test_null_context_is_rejected_without_touching_the_device(lib):
    assert lib.gw_grad(None, None, None, None, None, None, 0, None) == L.GW_ERR_INVALID
    assert lib.gw_ctx_check(None, None) == L.GW_ERR_INVALID
    assert lib.gw_last_error(None) == b"no context"


@pytest.mark.parametrize("cname,pytype", [("gw_problem", "gw_problem"),
                                           ("gw_barycenter_problem", "gw_barycenter_problem")])
def test_problem_struct_layout_matches_header(tmp_path, cname, pytype):
    """Offsets of the descriptor structs as the C compiler lays them out ==
    the ctypes mirrors."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    py = getattr(L, pytype)
    fields = [f for f, _ in py._fields_]
    src = tmp_path / "layout.c"
    body = "".join(f'  printf("%zu\\n", offsetof({cname}, {f}));\n' for f in fields)
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "gw.h"\nint main(void){\n'
                   + body + f'  printf("%zu\\n", sizeof({cname}));\n  return 0;\n}}\n')
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(L.ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    want = [getattr(py, f).offset for f in fields] + [ctypes.sizeof(py)]
    assert out == want
