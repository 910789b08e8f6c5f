"""The C ABI library builds for sm_103a, loads, and exports every entry point of include/*.h.

No CUDA call is made here (this runs on machines without a GPU)."""

import ctypes
import glob
import os
import re

import pytest

from paper_2305_18643_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s+\**\s*(ed_[A-Za-z0-9_]+)\s*\(", src, re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def libpath():
    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("ed_cluster_create", "ed_cluster_destroy", "ed_ground_state", "ed_green", "ed_hpsi",
                 "ed_basis", "ed_hop_table", "ed_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_library_is_sm103a_only(libpath):
    """The build asks nvcc for sm_103a code only (no other architectures, no PTX fallback)."""
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_2305_18643_gb300 import ed
    monkeypatch.setattr(ed, "_lib", None)
    monkeypatch.setattr(ed._build, "LIB", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError):
        ed.lib()


def declared_signatures():
    """{name: [parameter type strings]} of every function declared in include/*.h."""
    sigs = {}
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        for m in re.finditer(r"(ed_[A-Za-z0-9_]+)\s*\(([^;{]*?)\)\s*;", src, re.S):
            params = [p.strip() for p in m.group(2).split(",")]
            if params == ["void"] or params == [""]:
                params = []
            sigs[m.group(1)] = params
    return sigs


def _kind(ctype):
    """'ptr', 'f64', 'i64', 'i32' for a ctypes type; the same classes for a C parameter string."""
    import ctypes as C
    if ctype in (C.c_double,):
        return "f64"
    if ctype in (C.c_int64, C.c_uint64):
        return "i64"
    if ctype in (C.c_int, C.c_uint32, C.c_int32):
        return "i32"
    return "ptr"


def _ckind(param):
    if "*" in param:
        return "ptr"
    if param.startswith("double"):
        return "f64"
    if re.match(r"(u?int64_t|size_t|long)", param):
        return "i64"
    return "i32"


def test_binding_signatures_match_header(libpath):
    """Every entry point the Python binding declares has the header's parameter count and, slot by
    slot, the same class of type (pointer, double, 64-bit or 32-bit integer)."""
    from paper_2305_18643_gb300 import ed
    ed._lib = None
    lib = ed.lib()
    sigs = declared_signatures()
    checked = 0
    for name, params in sigs.items():
        f = getattr(lib, name)
        if f.argtypes is None:
            continue
        got = [_kind(t) for t in f.argtypes]
        want = [_ckind(p) for p in params]
        assert got == want, (name, got, want)
        checked += 1
    assert checked >= 15
