"""The Python binding's ctypes mirrors of the C-ABI structs (include/ww.h) have
the C layout: every field at the offset a C compiler gives it and every struct
of the same size.  A C program compiled against the header prints the layout;
no GPU and no library call is needed."""
import os
import shutil
import subprocess

import pytest

import paper_2609_36267_b300 as ww

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STRUCTS = [
    ("ww_params", ww.Params),
    ("ww_solve_stats", ww.SolveStats),
    ("ww_batch_item", ww.BatchItem),
    ("ww_server_config", ww.ServerConfig),
    ("ww_server_stats", ww.ServerStats),
    ("ww_tune_report", ww.TuneReport),
]


def _c_layout(tmp_path):
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "ww.h"', "int main(void) {"]
    for cname, cls in STRUCTS:
        lines.append(f'  printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for field, _ in cls._fields_:
            lines.append(f'  printf("{cname} {field} %zu\\n", offsetof({cname}, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                    str(exe)], check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    layout = {}
    for line in out.splitlines():
        cname, field, value = line.split()
        layout[(cname, field)] = int(value)
    return layout


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_ctypes_structs_match_the_c_layout(tmp_path):
    import ctypes

    layout = _c_layout(tmp_path)
    for cname, cls in STRUCTS:
        assert ctypes.sizeof(cls) == layout[(cname, "sizeof")], cname
        for field, _ in cls._fields_:
            assert getattr(cls, field).offset == layout[(cname, field)], (cname, field)
