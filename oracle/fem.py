"""Exact P1 stiffness on the blended mesh by element-wise assembly (IFEM).

Oracle (test infrastructure only; see the package docstring).

Paper, Sec. 2.2 (Eq. 2.3 and the algebraic system after it): the entries of
L_l are a_l(phi_I, phi_J) = <grad phi_I, grad phi_J> over Omega_l, the union of
the straight tetrahedra whose vertices are the Phi-mapped fine nodes.  Sec. 2.3:
every macro cell is refined regularly into N^3 tetrahedra (three congruence
classes); the stencil of an interior node couples it to 14 neighbours in the
named directions plus itself, and collects contributions from 24 tetrahedra.

Reading fixed here: the regular refinement is the Freudenthal-Kuhn
triangulation in the coordinates (alpha, beta, gamma) = (i + j + k, j + k, k):
every unit cube is cut into the six simplices x, x + e_s1, x + e_s1 + e_s2,
x + (1, 1, 1) that lie in N >= alpha >= beta >= gamma >= 0.  Its edge
directions in (i, j, k) are exactly the 14 offsets of DIRS below.
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp

from . import mesh as M

# The 15 cardinal directions of Sec. 2.3 (first letter: bottom / middle / top
# plane; rest: direction within the plane) as (i, j, k) offsets.  mc is the
# node itself.
DIR_NAMES = ("me", "mw", "mn", "ms", "mnw", "mse", "tc", "tw", "ts", "tse",
             "bc", "be", "bn", "bnw", "mc")
DIRS = np.array([
    (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (-1, 1, 0), (1, -1, 0),
    (0, 0, 1), (-1, 0, 1), (0, -1, 1), (1, -1, 1),
    (0, 0, -1), (1, 0, -1), (0, 1, -1), (-1, 1, -1), (0, 0, 0)], dtype=np.int64)
MC = 14


def kuhn_tets(N: int) -> np.ndarray:
    """The N^3 tetrahedra of the refined macro cell as (n, 4, 3) arrays of
    cell-local (i, j, k) vertex indices."""
    r = np.arange(N)
    org = np.stack(np.meshgrid(r, r, r, indexing="ij"), axis=-1).reshape(-1, 3)
    e = np.eye(3, dtype=np.int64)
    out = []
    for s in itertools.permutations(range(3)):
        v0 = org
        v1 = v0 + e[s[0]]
        v2 = v1 + e[s[1]]
        v3 = v0 + 1
        abg = np.stack([v0, v1, v2, v3], axis=1)           # (n, 4, 3) in (alpha, beta, gamma)
        ok = np.all((abg[..., 0] >= abg[..., 1]) & (abg[..., 1] >= abg[..., 2]) &
                    (abg[..., 2] >= 0) & (abg[..., 0] <= N), axis=1)
        abg = abg[ok]
        ijk = np.stack([abg[..., 0] - abg[..., 1], abg[..., 1] - abg[..., 2], abg[..., 2]], axis=-1)
        out.append(ijk)
    return np.concatenate(out, axis=0)


def element_stiffness(P: np.ndarray) -> np.ndarray:
    """Local P1 stiffness K_ab = |T| grad(lambda_a) . grad(lambda_b) of straight
    tetrahedra with vertices P (n, 4, 3); returns (n, 4, 4)."""
    E = P[:, 1:, :] - P[:, :1, :]                 # rows: edge vectors from vertex 0
    Einv = np.linalg.inv(E)                        # columns: gradients of lambda_1..3
    G = np.empty((len(P), 4, 3))
    G[:, 1:, :] = np.transpose(Einv, (0, 2, 1))
    G[:, 0, :] = -G[:, 1:, :].sum(axis=1)
    vol = np.abs(np.linalg.det(E)) / 6.0
    return vol[:, None, None] * np.einsum("nad,nbd->nab", G, G)


def cell_tet_nodes(N: int) -> np.ndarray:
    """Cell-local full-tet positions (lin_full) of the 4 vertices of every
    Kuhn tetrahedron, shape (N^3, 4)."""
    t = kuhn_tets(N)
    return M.lin_full(t[..., 0], t[..., 1], t[..., 2], N)


def assemble(level: M.Level, cells=None) -> sp.csr_matrix:
    """Global stiffness matrix L_l over all canonical nodes (Dirichlet rows
    and columns included), summed over the tetrahedra of `cells` (all cells
    by default)."""
    N = level.N
    loc = cell_tet_nodes(N)                         # (nT, 4)
    cells = np.arange(level.shell.nC) if cells is None else np.asarray(cells)
    rows, cols, vals = [], [], []
    for chunk in np.array_split(cells, max(1, len(cells) // 64)):
        glob = level.cell_map[chunk][:, loc]        # (nc, nT, 4)
        glob = glob.reshape(-1, 4)
        K = element_stiffness(level.coords[glob])
        rows.append(np.repeat(glob, 4, axis=1).ravel())
        cols.append(np.tile(glob, (1, 4)).ravel())
        vals.append(K.ravel())
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(level.n_total, level.n_total))
    return A.tocsr()


def interior_stencils(level: M.Level, A: sp.csr_matrix, cells=None) -> np.ndarray:
    """The 15 weights s_w (DIRS order) of every interior node of `cells`,
    read from the rows of A: shape (n_cells, n_l, 15)."""
    N = level.N
    cells = np.arange(level.shell.nC) if cells is None else np.asarray(cells)
    ip = M.interior_points(N)
    out = np.empty((len(cells), len(ip), 15))
    for n, c in enumerate(cells):
        row = level.cell_map[c][M.lin_full(ip[:, 0], ip[:, 1], ip[:, 2], N)]
        for w in range(15):
            q = ip + DIRS[w]
            col = level.cell_map[c][M.lin_full(q[:, 0], q[:, 1], q[:, 2], N)]
            out[n, :, w] = np.asarray(A[row, col]).ravel()
    return out


def free_block(A: sp.csr_matrix, level: M.Level) -> sp.csr_matrix:
    """A with the Dirichlet rows and columns removed (the unknowns only)."""
    f = level.free
    return A[f][:, f].tocsr()


def lumped_mass(level: M.Level) -> np.ndarray:
    """Vertex-quadrature weight of every canonical node: V_I = sum over the
    fine tetrahedra T containing node I of |T| / 4 (the row sums of the P1
    mass matrix).  Tetrahedra are straight with the level's node positions
    (mapped or not)."""
    loc = cell_tet_nodes(level.N)
    V = np.zeros(level.n_total)
    for chunk in np.array_split(np.arange(level.shell.nC), max(1, level.shell.nC // 64)):
        glob = level.cell_map[chunk][:, loc].reshape(-1, 4)
        P = level.coords[glob]
        vol = np.abs(np.linalg.det(P[:, 1:, :] - P[:, :1, :])) / 6.0
        for a in range(4):
            V += np.bincount(glob[:, a], weights=vol / 4.0, minlength=level.n_total)
    return V


def load_vector(level: M.Level, f_nodes: np.ndarray) -> np.ndarray:
    """Right-hand side of the accuracy study (Sec. 4): b_I = integral of f
    phi_I by the vertex quadrature rule on every tetrahedron, b_I = V_I f(x_I),
    for the unknowns; 0 at Dirichlet nodes."""
    b = np.zeros(level.n_total)
    fr = level.free
    b[fr] = lumped_mass(level)[fr] * f_nodes[fr]
    return b


def discretisation_error(level: M.Level, u_exact: np.ndarray, v: np.ndarray, H: float = 1.0) -> float:
    """e = h^(3/2) ||I_l(u) - v||_2 of Sec. 4.2 over all nodes, with
    h = H / N (Sec. 2.2: h_l = 2^-(l+2) H; the macro mesh size H is not
    given, 1 for the 60-cell shell and halved by each macro refinement).
    Its ratios (convergence orders, deviations from FEM) are pinned; its
    absolute values against Table 4.1 are parity unpinned (the paper's radii,
    macro mesh and H are not stated)."""
    return (H / level.N) ** 1.5 * float(np.linalg.norm(u_exact - v))
