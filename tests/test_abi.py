"""Host-side checks of the C ABI (no GPU needed): the library builds and loads,
exports every function include/plcg.h declares, and rejects bad arguments on
the host before any CUDA work."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_1905_06850_gb300 import build as B
from paper_1905_06850_gb300 import plcg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return plcg.load()


def header_functions():
    src = open(os.path.join(ROOT, "include", "plcg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(plcg_[a-z_0-9]+)\s*\(", src)))


def test_every_declared_symbol_is_exported_and_bound(lib):
    names = header_functions()
    assert len(names) >= 10
    for name in names:
        assert hasattr(lib, name), name
        assert name in plcg.SIGNATURES, name
    assert lib.plcg_version().decode().startswith("plcg")


def test_params_default(lib):
    p = plcg.plcg_params()
    lib.plcg_params_default(C.byref(p))
    assert p.l == 1 and p.rtol == 1e-8 and p.maxit == 100000 and p.max_restarts == 8
    assert p.prec == plcg.PLCG_FP64 and p.dots_2l1 == 0 and abs(p.inner_rtol_floor - 1e-4) < 1e-20
    assert p.precond == plcg.PLCG_PRECOND_NONE and p.grid_ctas == 0


def test_struct_layouts_match_header(tmp_path):
    """The ctypes structs have the sizes and field offsets gcc gives the
    header's structs."""
    import shutil
    import subprocess
    if not shutil.which("gcc"):
        pytest.skip("gcc not available")
    structs = {"plcg_params": plcg.plcg_params, "plcg_result": plcg.plcg_result,
               "plcg_stencil_desc": plcg.plcg_stencil_desc, "plcg_launch_info": plcg.plcg_launch_info}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "plcg.h"', 'int main(void) {']
    for name, st in structs.items():
        lines.append(f'printf("{name} %zu\\n", sizeof({name}));')
        for fname, _ in st._fields_:
            lines.append(f'printf("{name}.{fname} %zu\\n", offsetof({name}, {fname}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.run(["gcc", "-I", inc, str(src), "-o", str(exe)], check=True)
    got = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                       check=True).stdout.splitlines())
    for name, st in structs.items():
        assert int(got[name]) == C.sizeof(st), name
        for fname, _ in st._fields_:
            assert int(got[f"{name}.{fname}"]) == getattr(st, fname).offset, (name, fname)
    with pytest.raises(ValueError):
        plcg.make_params(precond="ilu")


@pytest.mark.parametrize("dim,points,nx,ny,nz", [(2, 7, 4, 4, 1), (3, 5, 4, 4, 4), (2, 5, 0, 4, 1),
                                                 (3, 7, 2048, 2048, 1024), (4, 9, 2, 2, 2)])
def test_bad_stencil_rejected_on_host(lib, dim, points, nx, ny, nz):
    d = plcg.plcg_stencil_desc(dim=dim, points=points, nx=nx, ny=ny, nz=nz, center=4.0, off=-1.0)
    h = C.c_void_p()
    assert lib.plcg_create_stencil(C.byref(d), None, C.byref(h)) == plcg.PLCG_ERR_INVALID
    assert not h.value
    assert "stencil" in plcg.last_error()


def test_bad_csr_rejected_on_host(lib):
    h = C.c_void_p()
    rowptr = np.array([0, 2, 1, 3], dtype=np.int64)        # decreasing
    col = np.array([0, 1, 2], dtype=np.int32)
    val = np.ones(3)
    st = lib.plcg_create_csr(3, 3, rowptr.ctypes.data, col.ctypes.data, val.ctypes.data, 0, 0,
                             None, C.byref(h))
    assert st == plcg.PLCG_ERR_INVALID and "rowptr" in plcg.last_error()
    rowptr = np.array([0, 1, 2, 3], dtype=np.int64)
    col = np.array([0, 5, 2], dtype=np.int32)               # out of range
    st = lib.plcg_create_csr(3, 3, rowptr.ctypes.data, col.ctypes.data, val.ctypes.data, 0, 0,
                             None, C.byref(h))
    assert st == plcg.PLCG_ERR_INVALID and "column" in plcg.last_error()
    col = np.array([0, 1, 2], dtype=np.int32)
    bad = np.array([1.0, np.nan, 1.0])
    st = lib.plcg_create_csr(3, 3, rowptr.ctypes.data, col.ctypes.data, bad.ctypes.data, 0, 0,
                             None, C.byref(h))
    assert st == plcg.PLCG_ERR_INVALID and "non-finite" in plcg.last_error()
    st = lib.plcg_create_csr(0, 0, rowptr.ctypes.data, None, None, 0, 0, None, C.byref(h))
    assert st == plcg.PLCG_ERR_INVALID


def test_null_arguments_rejected(lib):
    p = plcg.plcg_params()
    lib.plcg_params_default(C.byref(p))
    r = plcg.plcg_result()
    assert lib.plcg_solve(None, None, None, C.byref(p), C.byref(r)) == plcg.PLCG_ERR_INVALID
    assert lib.plcg_solve_host(None, None, None, C.byref(p), C.byref(r)) == plcg.PLCG_ERR_INVALID
    lib.plcg_destroy(None)


def test_binding_fails_loudly_without_library(tmp_path):
    import importlib
    mod = importlib.import_module("paper_1905_06850_gb300.plcg")
    saved = mod._lib
    try:
        mod._lib = None
        with pytest.raises(RuntimeError, match="missing"):
            mod.load(str(tmp_path / "nope.so"))
    finally:
        mod._lib = saved
