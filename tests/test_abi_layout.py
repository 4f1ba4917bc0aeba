"""The ctypes mirrors of the C-ABI structs (paper_1511_03645_gb300/adjamr.py)
against the header: a C program compiled from include/adjamr.h prints every
mirrored field's offset and every struct's size, which must equal the ctypes
layout (a field added to one side only, or out of order, shifts an offset or
the size).  CPU only: the header is plain C."""
import ctypes
import os
import shutil
import subprocess

import pytest

from paper_1511_03645_gb300 import adjamr as A

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MIRRORS = [
    ("adjamr_params", A.Params),
    ("adjamr_medium", A.Medium),
    ("adjamr_target", A.Target),
    ("adjamr_patch", A.Patch),
    ("adjamr_request", A.Request),
    ("adjamr_result", A.Result),
    ("adjamr_stats", A.Stats),
]


def _c_layout(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "adjamr.h"', "int main(void) {"]
    for cname, py in MIRRORS:
        lines.append(f'    printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'    printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True,
                   capture_output=True, text=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    layout = {}
    for line in out.splitlines():
        cname, key, val = line.split()
        layout[(cname, key)] = int(val)
    return layout


def test_ctypes_structs_match_the_header(tmp_path):
    layout = _c_layout(tmp_path)
    for cname, py in MIRRORS:
        assert ctypes.sizeof(py) == layout[(cname, "size")], cname
        for fname, _ in py._fields_:
            assert getattr(py, fname).offset == layout[(cname, fname)], f"{cname}.{fname}"
