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
