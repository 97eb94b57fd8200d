"""The C ABI's structs as the Python binding declares them (ctypes) against the header
(include/nlfeti.h) as a C compiler lays them out: every field the binding names exists in the
header's struct at the same offset, and the structs have the same size, so that a field added to
one side and not the other fails here instead of shifting the values the library reads.  Host
only (gcc)."""
import ctypes as C
import os
import shutil
import subprocess

import pytest

from paper_2306_00094_gb300 import binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PAIRS = {
    "Options": "nlfeti_options",
    "Stats": "nlfeti_stats",
    "Info": "nlfeti_info",
    "Profile": "nlfeti_profile",
    "ServerInfo": "nlfeti_server_info",
    "TuneEntry": "nlfeti_tune_entry",
    "Mesh": "nlfeti_mesh",
    "Kernel": "nlfeti_kernel",
    "Decomp": "nlfeti_decomp",
}


def _c_layout(tmp_path):
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "nlfeti.h"', "int main(void) {"]
    for py, c in PAIRS.items():
        lines.append(f'    printf("{py} size %zu\\n", sizeof({c}));')
        for name, _ in getattr(binding, py)._fields_:
            lines.append(f'    printf("{py} {name} %zu\\n", offsetof({c}, {name}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    r = subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    got = {}
    for line in out.splitlines():
        py, key, val = line.split()
        got[(py, key)] = int(val)
    return got


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_binding_structs_match_header(tmp_path):
    got = _c_layout(tmp_path)
    for py in PAIRS:
        cls = getattr(binding, py)
        assert got[(py, "size")] == C.sizeof(cls), (py, got[(py, "size")], C.sizeof(cls))
        for name, _ in cls._fields_:
            assert got[(py, name)] == getattr(cls, name).offset, (py, name)
