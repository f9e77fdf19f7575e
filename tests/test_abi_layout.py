"""The Python binding's ctypes structures against the C ABI's: a small C
program compiled with gcc against include/amr.h and include/amr_particles.h
prints the size of every struct and the offset of every field, and the
ctypes definitions must agree exactly (a field added on one side only would
let the library write past the binding's buffer)."""
import ctypes as C
import os
import shutil
import subprocess

import pytest

from paper_2607_20704_gb300 import amr

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STRUCTS = ["amr_params", "amr_member", "amr_info", "amr_server_params", "amr_request",
           "amr_server_stats", "amr_part_params", "amr_part_info"]


def _c_layout(tmp_path):
    if not shutil.which("gcc"):
        pytest.skip("no gcc")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "amr.h"', '#include "amr_particles.h"',
             'int main(void) {']
    for s in STRUCTS:
        lines.append(f'  printf("{s} size %zu\\n", sizeof({s}));')
        for f, _ in getattr(amr, s)._fields_:
            lines.append(f'  printf("{s} {f} %zu\\n", offsetof({s}, {f}));')
    lines += ['  return 0;', '}']
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    got = {}
    for line in out.splitlines():
        name, field, value = line.split()
        got[(name, field)] = int(value)
    return got


def test_ctypes_structs_match_the_header(tmp_path):
    c = _c_layout(tmp_path)
    for s in STRUCTS:
        cls = getattr(amr, s)
        assert C.sizeof(cls) == c[(s, "size")], (s, C.sizeof(cls), c[(s, "size")])
        for f, _ in cls._fields_:
            assert getattr(cls, f).offset == c[(s, f)], (s, f, getattr(cls, f).offset, c[(s, f)])
