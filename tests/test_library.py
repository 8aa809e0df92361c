"""The C-ABI library loads and exports every entry point include/hhg.h
declares (CPU only: no compute call)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "hhg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hhg_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared()
    for n in ("hhg_setup_shell", "hhg_fit_surrogate", "hhg_apply", "hhg_smooth", "hhg_residual", "hhg_vcycle",
              "hhg_destroy", "hhg_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol():
    import paper_1608_06473_gb300 as hhg
    if not os.path.exists(hhg.LIB_PATH):
        from paper_1608_06473_gb300 import _build
        _build.build()
    lib = ctypes.CDLL(hhg.LIB_PATH)
    for n in declared():
        assert hasattr(lib, n), n
    assert set(declared()) <= set(hhg.exported_symbols())
    assert hhg.hhg_last_error() == ""
