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


def test_problem_node_counts_match_the_mesh():
    """hhg_problem_nodes (host formula, no GPU): (N_r + 1)(10 n_t^2 + 2)
    nodes, the two boundary spheres Dirichlet -- against the oracle's mesh."""
    import paper_1608_06473_gb300 as hhg
    from oracle import mesh as M
    if not os.path.exists(hhg.LIB_PATH):
        from paper_1608_06473_gb300 import _build
        _build.build()
    for tang, layers, L in [(0, 1, 2), (0, 1, 4), (1, 2, 3), (2, 4, 3)]:
        sh = M.make_shell(tang=tang, layers=layers)
        lv = M.make_level(sh, 2 ** L)
        assert hhg.hhg_problem_nodes(0.45, 1.0, tang, layers, L) == (lv.n_total, len(lv.free))
    assert hhg.hhg_problem_nodes(0.55, 1.0, 2, 4, 6) == (168428034, 167117310)
    with pytest.raises(hhg.HHGError):
        hhg.hhg_problem_nodes(0.55, 1.0, 0, 1, 1)
