"""The ctypes mirrors of the C ABI's structs match include/tdvp.h field by field:
a small C program built with the host compiler prints sizeof and offsetof of
tdvp_opts and tdvp_request, and the binding's Structure classes must agree (a
mismatch would pass wrong values silently)."""
import ctypes as C
import os
import shutil
import subprocess

import pytest

from paper_2606_04771_b300._lib import Opts, RequestC

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

FIELDS = {
    "tdvp_opts": (Opts, ["precision", "krylov_max", "krylov_tol", "timeout_ms", "cuda_stream", "device",
                         "trunc_degeneracy", "merge_launches"]),
    "tdvp_request": (RequestC, ["L", "J", "U", "symmetry", "precision", "mode", "dt", "t_final", "chi_max", "eps",
                                "occupations"]),
}


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs a host C compiler")
def test_struct_layouts_match_the_header(tmp_path):
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "tdvp.h"', "int main(void) {"]
    for cname, (_, fields) in FIELDS.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for f in fields:
            lines.append(f'  printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for line in out:
        if line.strip():
            parts = line.split()
            got[tuple(parts[:-1])] = int(parts[-1])
    for cname, (cls, fields) in FIELDS.items():
        assert got[(cname, "size")] == C.sizeof(cls), cname
        for f in fields:
            assert got[(cname, f)] == getattr(cls, f).offset, (cname, f)


def test_binding_argument_counts_match_the_prototypes():
    import re

    from paper_2606_04771_b300._lib import lib

    text = open(os.path.join(ROOT, "include", "tdvp.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    protos = re.findall(r"\b(?:int|void|const char\s*\*)\s+(tdvp_\w+)\s*\(([^)]*)\)\s*;", text)
    assert len(protos) > 30
    L = lib()
    for name, args in protos:
        args = args.strip()
        n = 0 if args in ("", "void") else args.count(",") + 1
        f = getattr(L, name)
        assert f.argtypes is not None and len(f.argtypes) == n, (name, n, f.argtypes)
