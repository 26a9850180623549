"""The ctypes mirrors of the public structs match include/rbfkr.h field by field.

Each `typedef struct { ... } name;` of the header is parsed for its field
names in order, and a small C program built with the host compiler from the
header prints sizeof and every offsetof; the binding's ctypes classes must
have the same names, offsets and sizes (a field added on one side only would
otherwise shift every later field the library reads).
"""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rbfkr.h")

# header struct -> binding class name; the binding renames the field `lambda`
CLASSES = {"rbf_options": "Options", "rbf_operator": "Operator", "rbf_gkb_state": "GkbState",
           "rbf_solve_info": "SolveInfo", "rbf_timings": "Timings", "rbf_counters": "Counters",
           "rbf_batch": "Batch", "rbf_tuning": "Tuning", "rbf_stopnet": "StopNet",
           "rbf_learned_info": "LearnedInfo"}
RENAMED = {"lambda": "lambda_"}


def header_structs():
    txt = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    out = {}
    for body, name in re.findall(r"typedef\s+struct\s*\{(.*?)\}\s*(\w+)\s*;", txt, flags=re.S):
        fields = []
        for decl in body.split(";"):
            decl = decl.strip()
            if not decl:
                continue
            # "type a, b" / "type* p" / "type arr[2]": the declarators after the type
            head, *rest = decl.split(",")
            declarators = [head.split()[-1]] + [r.strip() for r in rest]
            for d in declarators:
                fields.append(re.sub(r"\[.*\]", "", d).strip("* "))
        out[name] = fields
    return out


def test_header_structs_parse():
    s = header_structs()
    assert set(CLASSES) <= set(s)
    assert s["rbf_options"][-1] == "fma_products"
    assert s["rbf_stopnet"][6:8] == ["l_min", "l_max"]


@pytest.mark.parametrize("cname", sorted(CLASSES))
def test_binding_fields_match_header_names(cname):
    from paper_2511_09798_gb300 import rbfkr
    cls = getattr(rbfkr, CLASSES[cname])
    want = [RENAMED.get(f, f) for f in header_structs()[cname]]
    assert [f for f, *_ in cls._fields_] == want


def test_binding_offsets_and_sizes_match_the_c_compiler():
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    from paper_2511_09798_gb300 import build, rbfkr
    structs = header_structs()
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "rbfkr.h"', "int main(void) {"]
    for cname in sorted(CLASSES):
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f in structs[cname]:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["return 0;", "}"]
    outdir = os.path.join(build.OUTDIR, "abi_layout")
    os.makedirs(outdir, exist_ok=True)
    src, exe = os.path.join(outdir, "layout.c"), os.path.join(outdir, "layout")
    with open(src, "w") as fh:
        fh.write("\n".join(lines) + "\n")
    r = subprocess.run([cc, "-std=c11", "-I", os.path.dirname(HEADER), src, "-o", exe], capture_output=True,
                       text=True)
    assert r.returncode == 0, r.stderr
    got = {}
    for line in subprocess.run([exe], capture_output=True, text=True, check=True).stdout.splitlines():
        cname, key, val = line.split()
        got[(cname, key)] = int(val)
    for cname, pyname in CLASSES.items():
        cls = getattr(rbfkr, pyname)
        assert ctypes.sizeof(cls) == got[(cname, "size")], cname
        for f in structs[cname]:
            assert getattr(cls, RENAMED.get(f, f)).offset == got[(cname, f)], (cname, f)
