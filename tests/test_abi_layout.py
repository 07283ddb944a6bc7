"""The ctypes mirrors of the C ABI's structs (sdd_params, sdd_stats, sdd_server_params,
sdd_server_stats, sdd_mc_config) have the C layout: a C program compiled against include/sdd.h prints the
size of each struct and the offset of each field, and the binding's structures match them."""
import ctypes
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

STRUCTS = {"sdd_params": "SddParams", "sdd_stats": "SddStats", "sdd_server_params": "SddServerParams",
           "sdd_server_stats": "SddServerStats", "sdd_mc_config": "SddMcConfig"}


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


def test_binding_argument_counts_match_the_prototypes():
    import re
    import paper_1504_00084_gb300 as S
    text = open(os.path.join(ROOT, "include", "sdd.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    protos = dict((m.group(1), m.group(2)) for m in re.finditer(r"\b(sdd_[a-z_0-9]+)\s*\(([^;{]*?)\)\s*;", text))
    assert protos
    checked = 0
    for name, params in protos.items():
        fn = getattr(S.lib, name)
        if fn.argtypes is None:
            continue
        params = params.strip()
        n = 0 if params in ("", "void") else params.count(",") + 1
        assert len(fn.argtypes) == n, (name, len(fn.argtypes), n)
        checked += 1
    assert checked >= 30
