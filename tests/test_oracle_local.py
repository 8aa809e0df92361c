"""Pins of the oracle's single-cell assembly (oracle/local.py) to its global
assembly.  CPU only.

Sec. 2.3: the row of a cell-interior node couples it to its 14 neighbours
through the 24 tetrahedra around it, all inside its own macro cell, so the
row assembled from that cell alone must equal the row of the global matrix
(fem.assemble) -- and, for the surrogate, the row of L~ (lsqp.surrogate_operator
with the coefficients of lsqp.fit).  Rows of vertex, edge and face nodes
collect the tetrahedra of every cell that contains the node; node_rows sums
them over those cells and must equal the global row too.  A dropped or doubled
cell, a wrong column map or a surrogate taken from the wrong cell fails one of
these element-wise comparisons.
"""
import numpy as np
import pytest

import synthetic as S
from oracle import fem as F
from oracle import local as LO
from oracle import lsqp as LS
from oracle import mesh as M

_cache = {}


def _global(tang, layers, N, q=2, j=2):
    key = (tang, layers, N, q, j)
    if key not in _cache:
        sh = M.make_shell(0.55, 1.0, tang, layers)
        lv = M.make_level(sh, N)
        A = F.assemble(lv)
        coef = LS.fit(lv, A, q=q, j=j)
        Ls = LS.surrogate_operator(lv, A, coef, q)
        _cache[key] = (sh, lv, A.tocsr(), Ls.tocsr())
    return _cache[key]


def _row_dict(A, r):
    s, e = A.indptr[r], A.indptr[r + 1]
    return {int(c): float(v) for c, v in zip(A.indices[s:e], A.data[s:e])}


def _check_rows(A, rows, cols, W, rtol=1e-14):
    for n in range(len(rows)):
        g = _row_dict(A, int(rows[n]))
        loc = {}
        for w in range(15):
            loc[int(cols[n, w])] = loc.get(int(cols[n, w]), 0.0) + float(W[n, w])
        assert set(g) == set(loc), f"column set differs at row {rows[n]}"
        scale = max(abs(v) for v in g.values())
        for c, v in g.items():
            assert abs(loc[c] - v) <= rtol * scale, (rows[n], c, loc[c], v)


@pytest.mark.parametrize("tang,layers,N", [(0, 1, 8), (0, 1, 16), (1, 2, 8)])
@pytest.mark.parametrize("op", ["ifem", "lsqp"])
def test_interior_rows_equal_global_rows(tang, layers, N, op):
    """interior_rows(c) == the global row of every interior node of 6 seeded
    cells, same columns, to 1e-14 relative (IFEM: L of fem.assemble; LSQP:
    L~ of lsqp.surrogate_operator)."""
    sh, lv, A, Ls = _global(tang, layers, N)
    cells = S.sample(sh.nC, 6, seed=700 + N + tang)
    for c in cells:
        rows, cols, W = LO.interior_rows(sh, N, int(c), op)
        assert len(rows) == M.n_cell_nodes(N)
        assert np.array_equal(rows, lv.off_C + int(c) * M.n_cell_nodes(N) + np.arange(len(rows)))
        _check_rows(A if op == "ifem" else Ls, rows, cols, W)


def test_interior_rows_differ_between_cells():
    """The surrogate rows of two different cells differ (so a row taken from
    the wrong cell would fail the comparison above)."""
    sh, lv, A, Ls = _global(0, 1, 16)
    _, _, W0 = LO.interior_rows(sh, 16, 0, "lsqp")
    _, _, W1 = LO.interior_rows(sh, 16, 1, "lsqp")
    assert np.max(np.abs(W0 - W1)) > 1e-6 * np.max(np.abs(W0))


@pytest.mark.parametrize("op", ["ifem", "lsqp"])
def test_node_rows_equal_global_rows_every_lower_node(op):
    """node_rows == the global row of every vertex, edge and face node of the
    60-cell shell at N = 8 (exact rows in both operators, Sec. 3.4), plus a
    seeded sample of interior nodes (surrogate rows for op = 'lsqp')."""
    N = 8
    sh, lv, A, Ls = _global(0, 1, N)
    lower = list(range(lv.off_C))
    interior = [int(x) for x in lv.off_C + S.sample(lv.n_total - lv.off_C, 40, seed=71)]
    got = LO.node_rows(sh, N, lower + interior, op)
    B = A if op == "ifem" else Ls
    for n in lower + interior:
        g = _row_dict(B, n)
        assert set(g) == set(got[n]), f"column set differs at node {n}"
        scale = max(abs(v) for v in g.values())
        for c, v in g.items():
            assert abs(got[n][c] - v) <= 1e-14 * scale, (n, c, got[n][c], v)


def test_node_rows_collect_every_adjacent_cell():
    """A lower node's row from node_rows uses every cell that holds the node:
    dropping one cell's contribution changes the row (checked against the
    global matrix assembled without that cell), so the comparison above would
    see a missing cell."""
    N = 8
    sh, lv, A, _ = _global(0, 1, N)
    v = 0  # macro vertex 0: shared by several cells
    cells = [c for c in range(sh.nC) if v in set(int(x) for x in sh.cells[c])]
    assert len(cells) >= 3
    partial = F.assemble(lv, cells=[c for c in range(sh.nC) if c != cells[0]]).tocsr()
    full = _row_dict(A, v)
    part = _row_dict(partial, v)
    assert max(abs(full[c] - part.get(c, 0.0)) for c in full) > 1e-3 * max(abs(x) for x in full.values())
