"""The structures of the C-ABI as the Python binding declares them (ctypes) against the C
header: a small C program compiled with the host compiler against include/rci.h prints the
size of every structure and the offset and size of every field, and each must equal the
binding's.  A field added, dropped, retyped or reordered on one side only fails here, on the
CPU, before any call crosses the boundary."""
import ctypes as C
import os
import shutil
import subprocess

import pytest

from paper_2207_10701_gb300 import rci

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# binding structure -> C typedef
PAIRS = {
    "GridDescC": "rci_grid_desc",
    "ObjectiveC": "rci_objective",
    "LightC": "rci_light",
    "InfoC": "rci_info",
    "ServerDescC": "rci_server_desc",
    "RequestC": "rci_request",
    "ResultC": "rci_result",
    "ServerStatsC": "rci_server_stats",
    "ProfileC": "rci_profile",
    "PeaksC": "rci_peaks",
}


def _c_layouts(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "rci.h"', "int main(void) {"]
    for py, c in PAIRS.items():
        lines.append(f'  printf("{py} size %zu\\n", sizeof({c}));')
        for name, _ in getattr(rci, py)._fields_:
            lines.append(f'  printf("{py} {name} %zu %zu\\n", offsetof({c}, {name}), '
                         f"sizeof((({c}*)0)->{name}));")
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    sizes, fields = {}, {}
    for ln in out.splitlines():
        parts = ln.split()
        if parts[1] == "size":
            sizes[parts[0]] = int(parts[2])
        else:
            fields[(parts[0], parts[1])] = (int(parts[2]), int(parts[3]))
    return sizes, fields


def test_every_binding_structure_matches_the_header(tmp_path):
    sizes, fields = _c_layouts(tmp_path)
    for py in PAIRS:
        cls = getattr(rci, py)
        assert C.sizeof(cls) == sizes[py], (py, C.sizeof(cls), sizes[py])
        for name, ctype in cls._fields_:
            off, size = fields[(py, name)]
            assert getattr(cls, name).offset == off, (py, name)
            assert C.sizeof(ctype) == size, (py, name)
