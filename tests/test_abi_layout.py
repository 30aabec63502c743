"""The ctypes mirrors of the C ABI's parameter structs (paper_1011_0911_gb300/lqcd.py)
against the header itself: a small C program compiled with the host compiler
prints sizeof and offsetof of every field, and each must equal the ctypes
layout.  A field added to one side only would shift every later field."""
import ctypes as C
import os
import shutil
import subprocess

import pytest

from paper_1011_0911_gb300 import lqcd

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# C typedef name -> ctypes mirror
PAIRS = [
    ("lqcd_geom", lqcd.Geom),
    ("lqcd_sap_params", lqcd.SapParams),
    ("lqcd_dfl_params", lqcd.DflParams),
    ("lqcd_solver_params", lqcd.SolverParams),
    ("lqcd_solve_info", lqcd.SolveInfo),
    ("lqcd_net_desc", lqcd.NetDesc),
    ("lqcd_net_train_params", lqcd.NetTrainParams),
    ("lqcd_block_params", lqcd.BlockParams),
    ("lqcd_md_params", lqcd.MDParams),
    ("lqcd_batch_params", lqcd.BatchParams),
]


def _c_program():
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "lqcd.h"', "int main(void) {"]
    for cname, cls in PAIRS:
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for f in cls._fields_:
            name = f[0]
            lines.append(f'  printf("{cname} {name} %zu\\n", offsetof({cname}, {name}));')
    lines += ["  return 0;", "}"]
    return "\n".join(lines) + "\n"


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    d = tmp_path_factory.mktemp("abi")
    src, exe = d / "layout.c", d / "layout"
    src.write_text(_c_program())
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    table = {}
    for line in out.splitlines():
        cname, field, value = line.split()
        table[(cname, field)] = int(value)
    return table


@pytest.mark.parametrize("cname,cls", PAIRS, ids=[p[0] for p in PAIRS])
def test_ctypes_mirror_matches_header(c_layout, cname, cls):
    assert C.sizeof(cls) == c_layout[(cname, "size")]
    for f in cls._fields_:
        assert getattr(cls, f[0]).offset == c_layout[(cname, f[0])], (cname, f[0])
