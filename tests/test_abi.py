"""C-ABI boundary checks that need no GPU: the library builds, loads, and
exports every entry point that include/lfe.h declares."""
import ctypes
import os
import re

import pytest

from paper_2608_12691_b300 import build as B
from paper_2608_12691_b300 import lfe

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "lfe.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lfe_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return ctypes.CDLL(B.LIB)


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 17
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(lfe.EXPORTED)


def test_binding_structs_match_header():
    # the ctypes mirrors carry every field of the C structs, in order
    src = open(os.path.join(ROOT, "include", "lfe.h")).read()
    body = src[src.index("typedef struct {", src.index("LFE_T_HB")):src.index("} lfe_params;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"([A-Za-z_0-9]+)(?:\[\d\])?\s*[;,]", body)
    assert [f[0] for f in lfe.Params._fields_] == fields


def test_create_without_gpu_reports_error():
    # on a machine without a GPU the library loads and lfe_create fails cleanly
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    from paper_2608_12691_b300 import systems as S
    d = S.make_water_box(seed=1, n_waters=20, box_len=1.2, solute=None, n_side=3, r_cut=0.55, grid=16)
    with pytest.raises(lfe.LfeError) as e:
        lfe.System(d)
    assert e.value.code == lfe.LFE_ERR_CUDA


def _header_signatures():
    src = open(os.path.join(ROOT, "include", "lfe.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    sigs = {}
    for ret, name, args in re.findall(r"([A-Za-z_][A-Za-z_0-9 ]*\**)\s*\b(lfe_[a-z_0-9]+)\s*\(([^()]*)\)\s*;",
                                      src):
        args = args.strip()
        sigs[name] = (ret.split()[-1] if ret.strip() else ret,
                      [] if args in ("", "void") else [a.strip() for a in args.split(",")])
    return sigs


def _c_kind(decl):
    if "*" in decl or "[" in decl:
        return "ptr"
    if "unsigned long long" in decl:
        return "u64"
    if "double" in decl:
        return "f64"
    if re.search(r"\bint\b", decl):
        return "i32"
    raise AssertionError(decl)


def _ctypes_kind(t):
    if t in (ctypes.c_void_p, ctypes.c_char_p) or (isinstance(t, type) and issubclass(t, ctypes._Pointer)):
        return "ptr"
    return {ctypes.c_double: "f64", ctypes.c_int: "i32", ctypes.c_ulonglong: "u64"}[t]


def test_binding_argument_types_match_header():
    # every entry point the binding calls is marshalled with the header's
    # argument count and kinds (pointer, int, double, 64-bit unsigned)
    sigs = _header_signatures()
    lib = lfe.load()
    assert set(sigs) == set(lfe.EXPORTED)
    for name, (ret, params) in sigs.items():
        fn = getattr(lib, name)
        assert fn.argtypes is not None, name
        assert [_ctypes_kind(t) for t in fn.argtypes] == [_c_kind(p) for p in params], name
        want = {"int": ctypes.c_int, "void": None, "char*": ctypes.c_char_p, "*": ctypes.c_char_p}[ret]
        assert fn.restype == want, (name, ret, fn.restype)


def test_struct_offsets_match_the_c_compiler(tmp_path):
    # the C compiler's offsets and sizes of lfe_params and lfe_topology equal
    # those of the ctypes mirrors (field order, types and padding)
    import subprocess
    structs = {"lfe_params": lfe.Params, "lfe_topology": lfe.Topology}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "lfe.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = {}
    for row in subprocess.check_output([str(exe)], text=True).split("\n"):
        if row:
            c, f, v = row.split()
            got[(c, f)] = int(v)
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)
