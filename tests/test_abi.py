"""CPU checks of the C ABI: the library builds for sm_103a, loads, and exports every entry point that
include/drt.h declares; the binding refuses to run without the library (no fallback)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "drt.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(drt_[A-Za-z_0-9]+)\s*\(", src)))


def test_header_declares_the_hot_path_calls():
    syms = declared_symbols()
    for name in ("drt_load_paths", "drt_extrapolate", "drt_synthesize_H", "drt_create", "drt_destroy"):
        assert name in syms


def test_library_builds_and_exports_every_declared_symbol():
    from paper_2205_00237_gb300 import build, drt
    path = build.build()
    lib = ctypes.CDLL(path)
    for name in declared_symbols():
        assert hasattr(lib, name), name
    assert sorted(drt.EXPORTS) == declared_symbols()


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_2205_00237_gb300 import drt
    with pytest.raises(RuntimeError):
        drt.load_library.__wrapped__(str(tmp_path / "missing.so")) if hasattr(drt.load_library, "__wrapped__") \
            else _load_missing(drt, tmp_path)


def _load_missing(drt, tmp_path):
    saved = drt._lib
    drt._lib = None
    try:
        drt.load_library(str(tmp_path / "missing.so"))
    finally:
        drt._lib = saved


def signatures():
    """{name: (return type, [parameter declarations])} of every function include/drt.h declares."""
    src = open(os.path.join(ROOT, "include", "drt.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    out = {}
    for m in re.finditer(r"(\w[\w\s\*]*?)\b(drt_[A-Za-z_0-9]+)\s*\(([^;{]*?)\)\s*;", src, flags=re.S):
        params = [p.strip() for p in " ".join(m.group(3).split()).split(",")]
        out[m.group(2)] = (m.group(1).strip(), [p for p in params if p and p != "void"])
    return out


def _ctype(decl):
    if "*" in decl or "[" in decl:
        return ctypes.c_void_p
    if decl.startswith("double"):
        return ctypes.c_double
    if "int64_t" in decl:
        return ctypes.c_uint64
    return ctypes.c_int32


def test_signatures_cover_every_declared_symbol():
    assert sorted(signatures()) == declared_symbols()


def test_every_entry_point_rejects_a_null_context():
    """Each status-returning call checks its context (and required outputs) before touching the device:
    with NULL it returns DRT_EINVAL and leaves a message, on any host, GPU or not."""
    from paper_2205_00237_gb300 import build
    lib = ctypes.CDLL(build.build())
    lib.drt_last_error.restype = ctypes.c_char_p
    checked = 0
    for name, (ret, params) in signatures().items():
        if ret != "drt_status":
            continue
        f = getattr(lib, name)
        types = [_ctype(p) for p in params]
        f.argtypes = types
        f.restype = ctypes.c_int32
        args = [None if t is ctypes.c_void_p else t(0) for t in types]
        assert f(*args) == -1, name
        assert lib.drt_last_error(), name
        checked += 1
    assert checked >= 25


def test_context_creation_fails_loudly_without_a_device():
    """No CPU fallback: without a CUDA device the library refuses to create a context."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    from paper_2205_00237_gb300 import build
    lib = ctypes.CDLL(build.build())
    lib.drt_last_error.restype = ctypes.c_char_p
    lib.drt_create.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint64]
    out = ctypes.c_void_p()
    assert lib.drt_create(ctypes.byref(out), 0, 0) == -3   # DRT_ECUDA
    assert out.value is None
    assert b"CUDA" in lib.drt_last_error()
