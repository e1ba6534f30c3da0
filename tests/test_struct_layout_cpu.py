"""The Python binding's ctypes mirrors of the C ABI's structs have the C layout: every
field's offset and every struct's size as gcc lays out include/vamrt.h (the same layout
nvcc's host compiler gives the library).  A field added on one side only, or in a
different order, fails here before any GPU call."""
import ctypes
import os
import shutil
import subprocess
import tempfile

import pytest

from paper_2211_03516_gb300 import vamrt as V

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
MIRRORS = {"vamrt_surface": V.Surface, "vamrt_geometry": V.Geometry, "vamrt_info": V.Info,
           "vamrt_opt_params": V.OptParams, "vamrt_opt_report": V.OptReport}


def _c_layout():
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ['#include "vamrt.h"', "#include <stdio.h>", "#include <stddef.h>", "int main(void) {"]
    for cname, py in MIRRORS.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for field, _ in py._fields_:
            lines.append(f'printf("{cname} {field} %zu\\n", offsetof({cname}, {field}));')
    lines += ["return 0;", "}"]
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "layout.c"), os.path.join(d, "layout")
        open(src, "w").write("\n".join(lines) + "\n")
        subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), src, "-o", exe], check=True,
                       capture_output=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    layout = {}
    for ln in out.splitlines():
        name, key, val = ln.split()
        layout[(name, key)] = int(val)
    return layout


@pytest.mark.parametrize("cname", list(MIRRORS))
def test_ctypes_mirror_matches_the_header(cname):
    layout = _c_layout()
    py = MIRRORS[cname]
    assert ctypes.sizeof(py) == layout[(cname, "size")]
    for field, _ in py._fields_:
        assert getattr(py, field).offset == layout[(cname, field)], field
