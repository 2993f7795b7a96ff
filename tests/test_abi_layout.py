"""The ctypes structures of the Python binding have the sizes and field offsets
that a C compiler gives the structures of include/tpp.h (host gcc; no GPU)."""
import ctypes
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

STRUCTS = {
    "tpp_problem": "Problem",
    "tpp_gmres_opts": "GmresOpts",
    "tpp_gmres_result": "GmresResult",
    "tpp_build_report": "BuildReport",
    "tpp_views": "Views",
    "tpp_batch_opts": "BatchOpts",
    "tpp_sys_problem": "SysProblem",
    "tpp_batch_report": "BatchReport",
    "tpp_time_report": "TimeReport",
}


def _c_layout():
    from paper_1704_04549_gb300 import _lib as L
    gcc = shutil.which("gcc") or shutil.which("cc")
    if gcc is None:
        pytest.skip("no host C compiler")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "tpp.h"', "int main(void) {"]
    for cname, pyname in STRUCTS.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for field, _ in getattr(L, pyname)._fields_:
            lines.append(f'  printf("{cname} {field} %zu\\n", offsetof({cname}, {field}));')
    lines += ["  return 0;", "}"]
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "layout.c"), os.path.join(d, "layout")
        open(src, "w").write("\n".join(lines) + "\n")
        subprocess.run([gcc, "-std=c11", "-I", os.path.join(ROOT, "include"), src, "-o", exe],
                       check=True, capture_output=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    table = {}
    for line in out.splitlines():
        name, key, val = line.split()
        table[(name, key)] = int(val)
    return table


def test_binding_structs_match_the_header():
    from paper_1704_04549_gb300 import _lib as L
    c = _c_layout()
    for cname, pyname in STRUCTS.items():
        cls = getattr(L, pyname)
        assert ctypes.sizeof(cls) == c[(cname, "size")], cname
        for field, _ in cls._fields_:
            assert getattr(cls, field).offset == c[(cname, field)], (cname, field)
