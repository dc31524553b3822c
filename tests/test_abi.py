"""The C ABI library loads and exports every function include/tmamg.h declares (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tmamg.h")


def declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tmamg_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_entry_points():
    names = declared()
    assert "tmamg_create" in names and "tmamg_dirac" in names


def test_library_exports_all_declared_symbols():
    from paper_2201_03872_gb300 import tmamg as T
    if not os.path.exists(T.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    lib = ctypes.CDLL(T.LIB_PATH)
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing
    # the Python binding wraps every declared entry point under the same name
    assert set(declared()) <= set(T.SIGNATURES), set(declared()) - set(T.SIGNATURES)


def test_binding_refuses_without_library(tmp_path, monkeypatch):
    from paper_2201_03872_gb300 import tmamg as T
    monkeypatch.setattr(T, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(T, "_lib", None)
    with pytest.raises(ImportError):
        T.lib()
