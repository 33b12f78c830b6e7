"""The ctypes structures of the binding lay out exactly like the C structures
of include/tomo.h: a host C compiler reports every structure's size and every
field's offset, and the binding must agree (a field added on one side only, or
out of order, would shift every later field silently)."""
import ctypes
import os
import shutil
import subprocess
import tempfile

import pytest

from paper_1302_3734_gb300 import binding as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PAIRS = [
    (B.Wfs, "tomo_wfs"),
    (B.Layer, "tomo_layer"),
    (B.Geometry, "tomo_geometry"),
    (B.PlanInfo, "tomo_plan_info"),
    (B.PlanOptions, "tomo_plan_options"),
    (B.Dm, "tomo_dm"),
    (B.FitGeometry, "tomo_fit_geometry"),
    (B.FitInfo, "tomo_fit_info"),
    (B.FrameResult, "tomo_frame_result"),
    (B.ServerStats, "tomo_server_stats"),
]


def _c_layout():
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "tomo.h"', "int main(void) {"]
    for cls, cname in PAIRS:
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in cls._fields_:
            lines.append(f'  printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["  return 0;", "}"]
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "layout.c"), os.path.join(d, "layout")
        with open(src, "w") as fh:
            fh.write("\n".join(lines) + "\n")
        subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), src, "-o", exe], check=True,
                       capture_output=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    layout = {}
    for line in out.splitlines():
        name, key, value = line.split()
        layout[(name, key)] = int(value)
    return layout


def test_binding_structures_match_the_header():
    layout = _c_layout()
    for cls, cname in PAIRS:
        assert ctypes.sizeof(cls) == layout[(cname, "size")], cname
        for f, _ in cls._fields_:
            assert getattr(cls, f).offset == layout[(cname, f)], (cname, f)
