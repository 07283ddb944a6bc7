"""The ctypes mirrors of the C ABI's structs (sdd_params, sdd_stats, sdd_server_params,
sdd_server_stats) have the C layout: a C program compiled against include/sdd.h prints the
size of each struct and the offset of each field, and the binding's structures match them."""
import ctypes
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

STRUCTS = {"sdd_params": "SddParams", "sdd_stats": "SddStats", "sdd_server_params": "SddServerParams",
           "sdd_server_stats": "SddServerStats"}


def test_struct_layouts_match_the_header(tmp_path):
    import paper_1504_00084_gb300 as S
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "sdd.h"', "int main(void) {"]
    for cname, pyname in STRUCTS.items():
        lines.append(f'    printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for field, _ in getattr(S, pyname)._fields_:
            lines.append(f'    printf("{cname} {field} %zu\\n", offsetof({cname}, {field}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True,
                   capture_output=True, timeout=120)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True, timeout=60).stdout
    for line in out.splitlines():
        cname, field, value = line.split()
        cls = getattr(S, STRUCTS[cname])
        got = ctypes.sizeof(cls) if field == "sizeof" else getattr(cls, field).offset
        assert got == int(value), (cname, field, got, value)
