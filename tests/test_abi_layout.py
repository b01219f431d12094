"""The ctypes binding's structures against the C header's (no GPU): a small C
program compiled with the header prints the size of every public struct and
the offset of each field, which must equal the ctypes layout field by field."""
import ctypes as C
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (C type, ctypes class name in _capi)
STRUCTS = [("wm_geom_desc", "GeomDesc"), ("wm_nurbs_patch", "NurbsPatch"), ("wm_sample_desc", "SampleDesc"),
           ("wm_schedule", "Schedule"), ("wm_stats", "Stats")]


def test_structs_match_the_header(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    from paper_2605_24882_gb300 import _capi
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "wmfield.h"', "int main(void) {"]
    for ctype, py in STRUCTS:
        cls = getattr(_capi, py)
        lines.append('  printf("%s size %%zu\\n", sizeof(%s));' % (ctype, ctype))
        for name, _ in cls._fields_:
            lines.append('  printf("%s %s %%zu\\n", offsetof(%s, %s));' % (ctype, name, ctype, name))
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for ln in out:
        if ln.strip():
            t, f, v = ln.split()
            got[(t, f)] = int(v)
    for ctype, py in STRUCTS:
        cls = getattr(_capi, py)
        assert got[(ctype, "size")] == C.sizeof(cls), ctype
        for name, _ in cls._fields_:
            assert got[(ctype, name)] == getattr(cls, name).offset, (ctype, name)


def test_constants_match_the_header():
    # every WM_ integer constant of the binding has the header's value
    import re
    from paper_2605_24882_gb300 import _capi
    hdr = open(os.path.join(ROOT, "include", "wmfield.h")).read()
    defs = {m.group(1): int(m.group(2)) for m in re.finditer(r"#define (WM_[A-Z0-9_]+) \(?(-?\d+)\)?", hdr)}
    ours = {k: v for k, v in vars(_capi).items() if k.startswith("WM_") and isinstance(v, int)}
    assert ours, "no constants in the binding"
    for k, v in ours.items():
        assert k in defs, k
        assert defs[k] == v, (k, defs[k], v)
