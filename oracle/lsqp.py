"""Least-squares surrogate stencils (LSQP) and the surrogate operator L~_l.

Oracle (test infrastructure only; see the package docstring).

Paper, Sec. 3.2: for every macro cell, level l >= 1 and cardinal direction w,
the stencil weight s_w(i, j, k) is replaced by the polynomial of total degree
<= q that fits the exact weights in the least-squares sense on the sampling
set S_l = M_{m(l, j)}, m(l, j) = min{l, max{1, j}} (Eq. 3.3); the matrix A has
one row per sampling point and one column per basis function (m_q columns,
Eq. 3.2).  Sec. 3.4: interior rows of L_l are replaced by the evaluated
polynomials (Eq. 3.4); lower-primitive rows stay exact; level 0 is not
replaced.  The Lemma of Sec. 3.4 shows the fitted centre polynomial equals
minus the sum of the others.

Readings fixed here:
  * sampling points of S_l are the level-l nodes 2^(l-m) (i, j, k),
    (i, j, k) in I_m, carrying the exact level-l stencil (this reproduces the
    point counts of Table 4.3);
  * basis: monomials xi_i^a xi_j^b xi_k^c, a + b + c <= q, with xi = (i, j, k)/N;
  * the least-squares problem is solved by Householder QR (DGELS, the routine
    the paper names in Sec. 4.2.2, is QR based);
  * the centre weight is minus the sum of the 14 fitted off-centre weights at
    the node (the form Alg. 5.1 uses; equal to the fitted centre polynomial by
    the Lemma of Sec. 3.4).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from . import fem as F
from . import mesh as M


def n_coeffs(q: int) -> int:
    """m_q of Eq. 3.2."""
    return (q + 3) * (q + 2) * (q + 1) // 6


def monomials(q: int):
    """Exponent triples (a, b, c), a + b + c <= q."""
    return [(a, b, c) for d in range(q + 1) for c in range(d + 1) for b in range(d + 1 - c)
            for a in [d - b - c]]


def level_index(N: int) -> int:
    """Paper level l with N = 2^(l+2) intervals per macro edge."""
    l = int(np.log2(N)) - 2
    assert 4 * 2 ** l == N
    return l


def sample_points(l: int, j: int) -> np.ndarray:
    """Cell-local level-l indices of the sampling set S_l = M_{m(l,j)} (Eq. 3.3)."""
    m = min(l, max(1, j))
    return M.interior_points(4 * 2 ** m) * 2 ** (l - m)


def design_matrix(pts: np.ndarray, N: int, q: int) -> np.ndarray:
    """Rows: the basis functions evaluated at the points."""
    xi = pts / float(N)
    return np.column_stack([xi[:, 0] ** a * xi[:, 1] ** b * xi[:, 2] ** c for a, b, c in monomials(q)])


def exact_weights_at(level: M.Level, A: sp.csr_matrix, c: int, pts: np.ndarray) -> np.ndarray:
    """Exact weights s_w (15 directions, DIRS order) of L_l at cell-local
    interior points of cell c, read from the assembled matrix."""
    N = level.N
    cm = level.cell_map[c]
    row = cm[M.lin_full(pts[:, 0], pts[:, 1], pts[:, 2], N)]
    out = np.empty((len(pts), 15))
    for w in range(15):
        qq = pts + F.DIRS[w]
        col = cm[M.lin_full(qq[:, 0], qq[:, 1], qq[:, 2], N)]
        out[:, w] = np.asarray(A[row, col]).ravel()
    return out


def fit(level: M.Level, A: sp.csr_matrix, q: int = 2, j: int = 2, cells=None) -> np.ndarray:
    """Coefficients a_w of the least-squares polynomials for the 14 off-centre
    directions of every cell: shape (n_cells, 14, m_q), basis = monomials(q)."""
    N = level.N
    l = level_index(N)
    assert l >= 1, "the surrogate replaces stencils on levels l >= 1 only"
    pts = sample_points(l, j)
    cells = np.arange(level.shell.nC) if cells is None else np.asarray(cells)
    out = np.empty((len(cells), 14, n_coeffs(q)))
    for n, c in enumerate(cells):
        out[n] = fit_values(pts, N, q, exact_weights_at(level, A, c, pts)[:, :14])
    return out


def fit_ipoly(level: M.Level, A: sp.csr_matrix, cells=None, q: int = 2) -> np.ndarray:
    """IPOLY (Sec. 3.1): the polynomials of degree q interpolating the exact
    off-centre weights at the m_q points of ipoly_points (a square system,
    solved like the least-squares one); shape (n_cells, 14, m_q)."""
    N = level.N
    assert level_index(N) >= 1
    pts = ipoly_points(N, q)
    cells = np.arange(level.shell.nC) if cells is None else np.asarray(cells)
    out = np.empty((len(cells), 14, n_coeffs(q)))
    for n, c in enumerate(cells):
        out[n] = fit_values(pts, N, q, exact_weights_at(level, A, c, pts)[:, :14])
    return out


def fit_values(pts: np.ndarray, N: int, q: int, b: np.ndarray) -> np.ndarray:
    """argmin_z ||A z - b||_2 (Sec. 3.2) for every column of b (values at the
    sampling points), by Householder QR; returns (n_columns, m_q)."""
    Q, R = np.linalg.qr(design_matrix(pts, N, q))
    return sla.solve_triangular(R, Q.T @ b).T


def evaluate(coef: np.ndarray, pts: np.ndarray, N: int, q: int) -> np.ndarray:
    """Surrogate weights at cell-local points: the 14 polynomials evaluated
    directly, centre = minus their sum.  coef (n_cells, 14, m_q) ->
    (n_cells, n_pts, 15)."""
    V = design_matrix(pts, N, q)                    # (n_pts, m_q)
    s = np.einsum("pm,cwm->cpw", V, coef)
    return np.concatenate([s, -s.sum(axis=2, keepdims=True)], axis=2)


def surrogate_operator(level: M.Level, A: sp.csr_matrix, coef: np.ndarray, q: int) -> sp.csr_matrix:
    """L~_l: A with every cell-interior row replaced by the surrogate stencil
    (Sec. 3.4); rows of vertex, edge and face nodes are kept exact."""
    return with_interior_stencils(level, A, evaluate(coef, M.interior_points(level.N), level.N, q))


def with_interior_stencils(level: M.Level, A: sp.csr_matrix, S: np.ndarray) -> sp.csr_matrix:
    """A with the row of every cell-interior node replaced by the 15 weights
    S (n_cells, n_l, 15) in the named directions; lower rows kept."""
    N = level.N
    ip = M.interior_points(N)
    Ac = A.tocoo()
    keep = Ac.row < level.off_C
    rows, cols, vals = [Ac.row[keep]], [Ac.col[keep]], [Ac.data[keep]]
    for c in range(level.shell.nC):
        cm = level.cell_map[c]
        r = cm[M.lin_full(ip[:, 0], ip[:, 1], ip[:, 2], N)]
        for w in range(15):
            qq = ip + F.DIRS[w]
            rows.append(r)
            cols.append(cm[M.lin_full(qq[:, 0], qq[:, 1], qq[:, 2], N)])
            vals.append(S[c, :, w])
    B = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=A.shape)
    return B.tocsr()


def fit_errors(exact: np.ndarray, surrogate: np.ndarray):
    """e_w^2 and e_w^inf of Sec. 3.3 per cell and direction: inputs
    (n_cells, n_l, 15) -> two arrays (n_cells, 15)."""
    d = exact - surrogate
    return np.sqrt(np.mean(d * d, axis=1)), np.max(np.abs(d), axis=1)


def ipoly_points(N: int, q: int = 2) -> np.ndarray:
    """The IPOLY interpolation points of Sec. 3.1: the nodes of degree q of
    the macro cell shrunk to its interior (vertices (1,1,1), (N-3,1,1),
    (1,N-3,1), (1,1,N-3)), i.e. (1,1,1) + (N-4) (a,b,c)/q for a+b+c <= q.
    For q = 2 these are the ten points a = N - 3, b = N/2 - 1 listed below;
    where (N-4)/q is not an integer (q = 3 and N = 8, 32, 128) each
    coordinate is rounded to the nearest fine node (the paper states the
    points for q = 2 only)."""
    if q == 2:
        a, b = N - 3, N // 2 - 1
        return np.array([(1, 1, 1), (1, 1, a), (1, a, 1), (a, 1, 1), (1, 1, b), (1, b, 1), (b, 1, 1),
                         (1, b, b), (b, 1, b), (b, b, 1)], dtype=np.int64)
    node = lambda x: int(np.floor(1.0 + (N - 4) * x / q + 0.5))
    return np.array([(node(a), node(b), node(c)) for a in range(q + 1) for b in range(q + 1 - a)
                     for c in range(q + 1 - a - b)], dtype=np.int64)
