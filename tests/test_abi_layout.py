"""The ctypes mirrors in the Python binding have the layout of the C structs of ufe.h.

A small C program built against the header prints sizeof and offsetof of every
field; the binding's ctypes.Structure classes must agree field by field (a mismatch
would make the binding read or pass garbage without any error).
"""
import ctypes
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

STRUCTS = {
    "ufe_mesh_info": "MeshInfo",
    "ufe_bddc_opts": "BddcOpts",
    "ufe_bddc_info": "BddcInfo",
    "ufe_solve_opts": "SolveOpts",
    "ufe_solve_info": "SolveInfo",
}


@pytest.mark.skipif(shutil.which("gcc") is None, reason="gcc not available")
@pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                    reason="nvcc not available")
def test_ctypes_structs_match_the_header(tmp_path):
    from paper_1703_06323_gb300 import build_ext
    build_ext.build()
    from paper_1703_06323_gb300 import ufe

    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "ufe.h"', "int main(void) {"]
    for cname, pyname in STRUCTS.items():
        cls = getattr(ufe, pyname)
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for field, _ in cls._fields_:
            lines.append(f'  printf("{cname} {field} %zu\\n", offsetof({cname}, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    c_layout = {}
    for line in out:
        if line:
            name, field, value = line.split()
            c_layout[name, field] = int(value)
    for cname, pyname in STRUCTS.items():
        cls = getattr(ufe, pyname)
        assert c_layout[cname, "size"] == ctypes.sizeof(cls), cname
        for field, _ in cls._fields_:
            assert c_layout[cname, field] == getattr(cls, field).offset, (cname, field)
