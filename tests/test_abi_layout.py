"""The ctypes structures of the binding against the C header's layout: a
small C program compiled with the host compiler prints sizeof and offsetof
of every field of every public structure, which must equal the binding's
(no GPU needed)."""
import ctypes as C
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STRUCTS = ("hz_params", "hz_frame_info", "hz_frame_desc", "hz_server_stats", "hz_profile")


def _c_name(field):
    return field[:-1] if field.endswith("_") else field  # `in_` stands for C's `in`


def test_binding_structs_match_the_header(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    from paper_2512_16609_gb300 import binding as b
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "hazedefy.h"', "int main(void) {"]
    for s in STRUCTS:
        lines.append(f'  printf("{s} size %zu\\n", sizeof({s}));')
        for f, _ in getattr(b, s)._fields_:
            lines.append(f'  printf("{s} {f} %zu\\n", offsetof({s}, {_c_name(f)}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    seen = 0
    for line in out:
        if not line.strip():
            continue
        s, f, v = line.split()
        cls = getattr(b, s)
        want = C.sizeof(cls) if f == "size" else getattr(cls, f).offset
        assert int(v) == want, (s, f, int(v), want)
        seen += 1
    assert seen == sum(1 + len(getattr(b, s)._fields_) for s in STRUCTS)
