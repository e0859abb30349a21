"""The ctypes structures of the binding against the C layout of include/kubo.h.

A C program compiled with the host compiler prints sizeof and offsetof of every field of the
ABI's structures; the binding's ctypes definitions must agree field by field, or options
would reach the library shifted.
"""
import ctypes
import json
import os
import shutil
import subprocess

import pytest

from paper_2309_06675_gb300 import BatchSchedule, Options, Problem, Profile

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

STRUCTS = {
    "kubo_profile": Profile,
    "kubo_options": Options,
    "kubo_problem": Problem,
    "kubo_batch_schedule": BatchSchedule,
}


def _c_layout(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "kubo.h"', 'int main(void) {',
             '  printf("{");']
    first = True
    for cname, py in STRUCTS.items():
        fields = ", ".join(
            f'\\"{f}\\": %zu' for f, _ in py._fields_)
        args = ", ".join(f"offsetof({cname}, {f})" for f, _ in py._fields_)
        sep = "" if first else ", "
        first = False
        lines.append(f'  printf("{sep}\\"{cname}\\": {{\\"sizeof\\": %zu, {fields}}}", '
                     f'sizeof({cname}), {args});')
    lines += ['  printf("}\\n");', '  return 0;', '}']
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    return json.loads(out)


def test_ctypes_structures_match_the_c_header(tmp_path):
    c = _c_layout(tmp_path)
    for cname, py in STRUCTS.items():
        assert c[cname]["sizeof"] == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert c[cname][f] == getattr(py, f).offset, (cname, f)
