"""The ctypes structures of the binding have the layout of the C ABI headers.

A small C program, compiled here with the host compiler against
include/pdas.h and include/pdas_batch.h, prints sizeof and offsetof of every
field the binding declares; each must match the ctypes structure.  This
catches a field added to a header but not to the binding (or the reverse)
without a GPU.
"""
import ctypes
import os
import shutil
import subprocess
import tempfile

import pytest

from paper_1502_03543_gb300 import _native as N

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INCLUDE = os.path.join(ROOT, "include")

# (C type name, ctypes structure)
STRUCTS = [
    ("pdas_options", N.Options),
    ("pdas_iter_info", N.IterInfo),
    ("pdas_profile", N.Profile),
    ("pdas_batch_options", N.BatchOptions),
]


def _c_layout():
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "pdas.h"', '#include "pdas_batch.h"',
             "int main(void) {"]
    for cname, st in STRUCTS:
        lines.append('  printf("%s sizeof %zu\\n", "{0}", sizeof({0}));'.replace("{0}", cname))
        for field, _ in st._fields_:
            lines.append('  printf("%s %s %zu\\n", "{0}", "{1}", offsetof({0}, {1}));'.replace("{0}", cname)
                         .replace("{1}", field))
    lines.append('  printf("stages %d\\n", (int)PDAS_STAGE_COUNT);')
    lines += ["  return 0;", "}"]
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "layout.c"), os.path.join(d, "layout")
        with open(src, "w") as f:
            f.write("\n".join(lines) + "\n")
        subprocess.run([cc, "-std=c11", "-I", INCLUDE, src, "-o", exe], check=True, capture_output=True, text=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    layout = {}
    for line in out.splitlines():
        parts = line.split()
        layout[tuple(parts[:-1])] = int(parts[-1])
    return layout


def test_structures_match_headers():
    layout = _c_layout()
    for cname, st in STRUCTS:
        assert ctypes.sizeof(st) == layout[(cname, "sizeof")], cname
        for field, _ in st._fields_:
            assert getattr(st, field).offset == layout[(cname, field)], (cname, field)
    # the profile's per-stage arrays and the binding's stage names
    assert layout[("stages",)] == len(N.STAGES) == dict(N.Profile._fields_)["ms"]._length_
