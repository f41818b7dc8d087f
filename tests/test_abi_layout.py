"""The ctypes structures of the binding have the C layout of include/fetirp.h: a small C program compiled
against the header prints every size and field offset, and the binding's structures must agree."""
import ctypes as C
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
F = pytest.importorskip("paper_1208_6387_gb300.fetirp")

STRUCTS = {"fetirp_options": F.fetirp_options, "fetirp_stats": F.fetirp_stats,
           "fetirp_structure": F.fetirp_structure}


def _c_layout():
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "fetirp.h"', "int main(void) {"]
    for name, cls in STRUCTS.items():
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'  printf("{name}.{field} %zu\\n", offsetof({name}, {field}));')
    lines += ["  return 0;", "}"]
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "layout.c"), os.path.join(d, "layout")
        with open(src, "w") as f:
            f.write("\n".join(lines) + "\n")
        subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), src, "-o", exe], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    return dict(line.rsplit(" ", 1) for line in out.splitlines())


def test_binding_structs_match_the_header():
    lay = _c_layout()
    for name, cls in STRUCTS.items():
        assert int(lay[f"{name} size"]) == C.sizeof(cls), name
        for field, _ in cls._fields_:
            assert int(lay[f"{name}.{field}"]) == getattr(cls, field).offset, (name, field)
