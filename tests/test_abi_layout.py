"""The C structs of include/drr.h and the Python binding's ctypes mirrors have the
same size and field offsets: a small C program built with the host compiler
against the header prints them (no GPU, no library call)."""
import ctypes
import os
import shutil
import subprocess

import pytest

from paper_2208_12737_gb300 import drr

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STRUCTS = ["drr_detector", "drr_volume_options", "drr_server_config", "drr_request", "drr_result",
           "drr_server_stats"]


def _c_layout(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "drr.h"', "int main(void) {"]
    for name in STRUCTS:
        cls = getattr(drr, name)
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'  printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    table = {}
    for line in out.splitlines():
        struct, key, value = line.split()
        table[(struct, key)] = int(value)
    return table


def test_ctypes_mirrors_match_the_header(tmp_path):
    c = _c_layout(tmp_path)
    for name in STRUCTS:
        cls = getattr(drr, name)
        assert ctypes.sizeof(cls) == c[(name, "size")], name
        for field, _ in cls._fields_:
            assert getattr(cls, field).offset == c[(name, field)], (name, field)
