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


def _c_kind(decl):
    """Kind of a C parameter or return type: ptr, f64, f32, or i/u with its width in bits."""
    d = " ".join(decl.split())
    if "*" in d or "[" in d:
        return "ptr"
    for words, kind in (("double", "f64"), ("float", "f32"), ("unsigned long long", "u64"), ("uint64_t", "u64"),
                        ("size_t", "u64"), ("long long", "i64"), ("int64_t", "i64"), ("uint32_t", "u32"),
                        ("unsigned", "u32"), ("int", "i32")):
        if re.search(r"\b" + words + r"\b", d):
            return kind
    raise AssertionError(f"unknown C type in {decl!r}")


def _ctypes_kind(t):
    if t is None:
        return "void"
    if t in (C.c_void_p, C.c_char_p) or issubclass(t, C._Pointer):
        return "ptr"
    if t is C.c_double:
        return "f64"
    if t is C.c_float:
        return "f32"
    signed = t(-1).value < 0
    return ("i" if signed else "u") + str(8 * C.sizeof(t))


def _prototypes():
    text = open(os.path.join(__graft_entry__.ROOT, "include", "polrt.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return re.findall(r"^\s*(int|size_t|long long|const char \*)\s*(rt_\w+)\s*\(([^;]*?)\)\s*;", text, re.M | re.S)


def test_binding_argument_types_match_the_prototypes():
    from paper_2302_02733_gb300 import build

    build.build()
    L = polrt.lib()
    protos = _prototypes()
    assert len(protos) >= 40
    for ret, name, args in protos:
        fn = getattr(L, name)
        params = [] if args.strip() == "void" else [a for a in args.split(",")]
        want = [_c_kind(a) for a in params]
        assert fn.argtypes is not None, f"{name}: no argtypes"
        assert [_ctypes_kind(t) for t in fn.argtypes] == want, name
        if ret == "const char *":
            assert _ctypes_kind(fn.restype) == "ptr", name
        else:
            assert _ctypes_kind(fn.restype) == _c_kind(ret), name
