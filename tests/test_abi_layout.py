"""CPU check that the ctypes binding describes the C ABI exactly: every structure the binding
declares has the size and the field offsets that a C compiler gives the same structure from
include/polrt.h, and every constant the binding defines has the header's value. A field left
out, reordered or given the wrong width in polrt.py would otherwise shift every later field
without an error. No GPU is used."""
import ctypes as C
import os
import re
import shutil
import subprocess
import tempfile

import pytest

import __graft_entry__  # noqa: F401  (puts the repo root on sys.path)

from paper_2302_02733_gb300 import polrt


def _structs():
    return {n: t for n, t in vars(polrt).items()
            if n.startswith("rt_") and isinstance(t, type) and issubclass(t, C.Structure)}


def _constants():
    return {n: v for n, v in vars(polrt).items() if re.fullmatch(r"RT_[A-Z0-9_]+", n) and isinstance(v, int)}


def _c_layout():
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "polrt.h"', "int main(void) {"]
    for name, t in sorted(_structs().items()):
        lines.append(f'    printf("size {name} %zu\\n", sizeof({name}));')
        for f in t._fields_:
            lines.append(f'    printf("off {name}.{f[0]} %zu\\n", offsetof({name}, {f[0]}));')
    for name in sorted(_constants()):
        lines.append(f'    printf("const {name} %lld\\n", (long long)({name}));')
    lines += ["    return 0;", "}"]
    inc = os.path.join(__graft_entry__.ROOT, "include")
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "layout.c"), os.path.join(d, "layout")
        with open(src, "w") as fh:
            fh.write("\n".join(lines) + "\n")
        r = subprocess.run([cc, "-std=c99", "-I", inc, "-o", exe, src], capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout
    got = {}
    for ln in out.splitlines():
        kind, key, val = ln.split()
        got[(kind, key)] = int(val)
    return got


def test_struct_sizes_and_offsets_match_the_header():
    got = _c_layout()
    structs = _structs()
    assert {"rt_camera", "rt_model_params", "rt_counters", "rt_job", "rt_batch_config",
            "rt_render_config", "rt_mlp_norm", "rt_batch_stats"} <= set(structs)
    for name, t in structs.items():
        assert C.sizeof(t) == got[("size", name)], name
        for f in t._fields_:
            assert getattr(t, f[0]).offset == got[("off", f"{name}.{f[0]}")], f"{name}.{f[0]}"


def test_constants_match_the_header():
    got = _c_layout()
    consts = _constants()
    assert len(consts) >= 25
    for name, v in consts.items():
        assert v == got[("const", name)], name
