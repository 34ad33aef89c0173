"""The binding's ctypes mirrors of the C ABI's structs against include/gapla.h:
the same fields in the same order, and, as gcc lays the header out, the same
offset for every field and the same size for every struct."""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

import paper_2507_13375_gb300 as la

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gapla.h")
STRUCTS = {"la_grid_desc": la.GridDesc, "la_net_desc": la.NetDesc, "la_round_params": la.RoundParams,
           "la_round_stats": la.RoundStats}


def header_fields():
    """{struct name: [field names in order]} of the header's typedef structs."""
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    out = {}
    for body, name in re.findall(r"typedef struct\s*\{(.*?)\}\s*(la_\w+)\s*;", text, flags=re.S):
        names = []
        for decl in body.split(";"):
            decl = re.sub(r"\[[^\]]*\]", "", decl).strip()
            if decl:  # one type, one or more declarators ("int32_t X, Y, L")
                names += [re.findall(r"[A-Za-z_]\w*", part)[-1] for part in decl.split(",")]
        out[name] = names
    return out


def test_fields_match_the_header():
    fields = header_fields()
    for cname, py in STRUCTS.items():
        assert [f for f, _ in py._fields_] == fields[cname], cname


def test_offsets_and_sizes_match_gcc(tmp_path):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no gcc")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "gapla.h"', "int main(void) {"]
    for cname, py in STRUCTS.items():
        lines.append(f'  printf("{cname} . %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines.append("  return 0;\n}")
    src, exe = tmp_path / "layout.c", tmp_path / "layout"
    src.write_text("\n".join(lines) + "\n")
    subprocess.run([gcc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        c, f, v = line.split()
        got[(c, f)] = int(v)
    for cname, py in STRUCTS.items():
        assert got[(cname, ".")] == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)
