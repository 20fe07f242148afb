"""The ctypes structures of the binding have the layout of the C structures in
include/sipf.h: a small C program built with the host compiler prints the
size of every structure and the offset of every field, and the binding's
ctypes classes must agree (no GPU needed)."""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

from paper_2512_03452_gb300 import _abi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INCLUDE = os.path.join(ROOT, "include")
STRUCTS = ["sipf_params", "sipf_diag", "sipf_timing", "sipf_batch_tuning"]


def _c_layout(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "sipf.h"', "int main(void) {"]
    for name in STRUCTS:
        cls = getattr(_abi, name)
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'  printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", INCLUDE, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    layout = {}
    for line in out.splitlines():
        name, key, val = line.split()
        layout[(name, key)] = int(val)
    return layout


def test_every_header_structure_is_bound():
    text = open(os.path.join(INCLUDE, "sipf.h")).read()
    defined = set(re.findall(r"typedef struct (\w+) \{", text))
    assert defined == set(STRUCTS)


def test_binding_structures_match_the_header(tmp_path):
    layout = _c_layout(tmp_path)
    for name in STRUCTS:
        cls = getattr(_abi, name)
        assert ctypes.sizeof(cls) == layout[(name, "size")], name
        for field, _ in cls._fields_:
            assert getattr(cls, field).offset == layout[(name, field)], (name, field)
