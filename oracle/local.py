"""Stencil rows of single macro cells, for sampled checks on large shells.

Oracle (test infrastructure only; see the package docstring).

Rows of cell-interior nodes involve only the 24 tetrahedra around the node,
all inside its macro cell (Sec. 2.3), so they can be assembled from that cell
alone: the same element-wise assembly as `fem.assemble`, restricted to one
cell's N^3 tetrahedra, and the same least-squares fit as `lsqp.fit`.  Shells
whose global matrix would not fit in host memory (3840 macro cells at N = 64)
are checked on a seeded sample of cells this way.
"""
from __future__ import annotations

import functools

import numpy as np
import scipy.sparse as sp

from . import fem as F
from . import lsqp as LS
from . import mesh as M


def _offsets(sh: M.Shell, N: int):
    return M._prim_offsets(sh, N)


@functools.lru_cache(maxsize=8)
def _tet_nodes(N: int) -> np.ndarray:
    """fem.cell_tet_nodes(N), computed once per N (the same for every cell)."""
    return F.cell_tet_nodes(N)


def cell_map(sh: M.Shell, N: int, c: int) -> np.ndarray:
    """Canonical index of every cell-local point (lin_full order)."""
    fp = M.full_points(N)
    return M.node_index(sh, N, np.tile(sh.cells[c], (len(fp), 1)), M.cell_lambda(N, fp), np.full(len(fp), c))


def cell_coords(sh: M.Shell, N: int, c: int) -> np.ndarray:
    """Mapped positions of every cell-local point (identical to the canonical
    positions of the same nodes, except the four macro vertices, which agree
    to an ulp)."""
    fp = M.full_points(N)
    return M.blend(sh, np.tile(sh.cells[c], (len(fp), 1)), M.cell_lambda(N, fp), N)


def cell_matrix(sh: M.Shell, N: int, c: int) -> sp.csr_matrix:
    """Sum of the element matrices of cell c's tetrahedra, in cell-local
    (lin_full) numbering; its interior rows are rows of L_l."""
    loc = _tet_nodes(N)
    X = cell_coords(sh, N, c)
    K = F.element_stiffness(X[loc])
    n = M.tet_count(N)
    A = sp.coo_matrix((K.ravel(), (np.repeat(loc, 4, axis=1).ravel(), np.tile(loc, (1, 4)).ravel())),
                      shape=(n, n))
    return A.tocsr()


def exact_stencils(sh: M.Shell, N: int, c: int, pts: np.ndarray) -> np.ndarray:
    """Exact 15 weights at cell-local interior points of cell c."""
    A = cell_matrix(sh, N, c)
    row = M.lin_full(pts[:, 0], pts[:, 1], pts[:, 2], N)
    out = np.empty((len(pts), 15))
    for w in range(15):
        qq = pts + F.DIRS[w]
        out[:, w] = np.asarray(A[row, M.lin_full(qq[:, 0], qq[:, 1], qq[:, 2], N)]).ravel()
    return out


def interior_rows(sh: M.Shell, N: int, c: int, op: str = "lsqp", q: int = 2, j: int = 2):
    """Rows of all interior nodes of cell c: canonical row indices (n_l,),
    canonical column indices (n_l, 15) and weights (n_l, 15), DIRS order.
    op = 'ifem' gives L_l, 'lsqp' the surrogate L~_l (exact on N = 4)."""
    ip = M.interior_points(N)
    cm = cell_map(sh, N, c)
    rows = cm[M.lin_full(ip[:, 0], ip[:, 1], ip[:, 2], N)]
    cols = np.stack([cm[M.lin_full(*(ip + F.DIRS[w]).T, N)] for w in range(15)], axis=1)
    if op == "lsqp" and N >= 8:
        l = LS.level_index(N)
        pts = LS.sample_points(l, j)
        coef = LS.fit_values(pts, N, q, exact_stencils(sh, N, c, pts)[:, :14])
        W = LS.evaluate(coef[None], ip, N, q)[0]
    else:
        W = exact_stencils(sh, N, c, ip)
    return rows, cols, W


def colour_of(N: int) -> np.ndarray:
    """Cell-interior colour (i + 2j + 3k) mod 4 of every interior point."""
    ip = M.interior_points(N)
    return (ip[:, 0] + 2 * ip[:, 1] + 3 * ip[:, 2]) % 4


def interior_colour_steps(rows, cols, W, colour, u, f):
    """Steps 7-10 of a sweep (cell-interior colours 0..3) restricted to one
    macro cell: Eq. 5.1 on every node of the colour from the values at the
    start of the step.  rows/cols index u and f (any numbering); u is
    updated in place and returned."""
    for cc in range(4):
        S = colour == cc
        acc = f[rows[S]].copy()
        for w in range(14):
            acc = acc - W[S, w] * u[cols[S, w]]
        u[rows[S]] = acc / W[S, 14]
    return u


def node_rows(sh: M.Shell, N: int, nodes, op: str = "ifem", q: int = 2, j: int = 2):
    """Rows of L_l (or L~_l for op='lsqp' at cell-interior nodes) for a list of
    canonical nodes of any primitive, assembled from the cells that contain
    them: {node: {column: weight}}.  Lower-primitive rows are exact in both
    operators (Sec. 3.4)."""
    cache = {}

    def cell(c):
        if c not in cache:
            cache[c] = (cell_map(sh, N, c), cell_matrix(sh, N, c))
        return cache[c]

    out = {}
    for n in nodes:
        verts = set(M.primitive_of(sh, N, n))
        row = {}
        for c in np.flatnonzero([verts <= set(int(x) for x in cv) for cv in sh.cells]):
            cm, A = cell(int(c))
            loc = np.flatnonzero(cm == n)
            if len(loc) == 0:
                continue
            r = A.getrow(int(loc[0]))
            for jj, a in zip(r.indices, r.data):
                row[int(cm[jj])] = row.get(int(cm[jj]), 0.0) + a
        out[n] = row
    off_C = M.offsets(sh, N)[2]
    if op == "lsqp" and N >= 8:
        for n in nodes:
            if n >= off_C:
                c = (n - off_C) // M.n_cell_nodes(N)
                rows, cols, W = interior_rows(sh, N, int(c), "lsqp", q, j)
                k = int(np.flatnonzero(rows == n)[0])
                out[n] = {int(cols[k, w]): float(W[k, w]) for w in range(15)}
    return out
