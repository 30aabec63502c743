"""Host-side checks of the C-ABI library: it builds for sm_103a, loads, and
exports every entry point include/lqcd.h declares.  No compute calls (no GPU
needed)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "lqcd.h")).read()
    return sorted(set(re.findall(r"LQCD_API[^;(]*?\b(lqcd_\w+)\s*\(", src)))


def test_header_declares_entry_points():
    names = declared_symbols()
    for must in ("lqcd_create", "lqcd_apply_D", "lqcd_apply_Dhat", "lqcd_clover_invert", "lqcd_dfl_build",
                 "lqcd_solve_dhat", "lqcd_sap"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_1011_0911_gb300 import build_lib
    path = build_lib.build()
    L = C.CDLL(path)
    missing = [n for n in declared_symbols() if not hasattr(L, n)]
    assert not missing, missing


def test_create_rejects_bad_geometry_without_touching_the_gpu():
    """lqcd_create validates the lattice before any CUDA call."""
    from paper_1011_0911_gb300 import lqcd
    L = lqcd.lib()
    h = C.c_void_p()
    for dims in ((3, 4, 4, 4), (4, 4, 4, 0), (4, -2, 4, 4)):
        g = lqcd.Geom(*dims, 1)
        assert L.lqcd_create(C.byref(g), None, C.byref(h)) == 1
        assert not h.value


def test_oracle_builds_and_loads():
    import oracle
    assert oracle.lib() is not None
