"""Macro mesh of the thick spherical shell, HHG primitives and fine nodes.

Oracle (test infrastructure only; see the package docstring).

Paper, Sec. 2.2: the domain is the shell r1 < |x| < r2 (Eq. 2.1); an
unstructured tetrahedral macro mesh T_{-2} is regularly refined (Bey), and the
nodes of every refined mesh are moved by a blending map Phi so that interior
macro layers become spherical.  Sec. 2.3: fine nodes are grouped into vertex,
edge, face and volume (cell) primitives; the interior nodes of a macro cell are
addressed by index triples (i, j, k) with i, j, k >= 1 and i + j + k <= N - 1,
where N = 2^(l+2) is the number of intervals per macro edge on level l.

Readings fixed here (the paper leaves them open):
  * macro mesh: icosahedron, t tangential 1:4 refinements projected to the
    unit sphere, M uniform radial layers between r1 and r2, every prism split
    into three tetrahedra by the vertex ids (conforming);
  * local vertex order of a macro cell = ascending global vertex id; i, j, k
    count along the local edges 0->1, 0->2, 0->3;
  * Phi(x) = rho(x) x/|x| with rho the linear interpolant of the radii of the
    macro cell's vertices;
  * canonical node order: vertices, then edges, then faces, then cells, each
    primitive's nodes in its local index order.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass, field

import numpy as np


# ----------------------------------------------------------------------------
# Macro mesh
# ----------------------------------------------------------------------------

def _unit(x: np.ndarray) -> np.ndarray:
    """Rows of x divided by their Euclidean length."""
    n = np.sqrt(x[:, 0] * x[:, 0] + x[:, 1] * x[:, 1] + x[:, 2] * x[:, 2])
    return x / n[:, None]


def icosahedron():
    """Unit icosahedron: 12 vertices (cyclic permutations of (0, +-1, +-g),
    g the golden ratio, normalised) and its 20 faces as ascending id triples,
    sorted lexicographically."""
    g = (1.0 + np.sqrt(5.0)) / 2.0
    raw = np.array([
        (0, -1, -g), (0, -1, g), (0, 1, -g), (0, 1, g),
        (-1, -g, 0), (-1, g, 0), (1, -g, 0), (1, g, 0),
        (-g, 0, -1), (-g, 0, 1), (g, 0, -1), (g, 0, 1)], dtype=np.float64)
    tris = []
    for a, b, c in itertools.combinations(range(12), 3):
        d = [np.sum((raw[p] - raw[r]) ** 2) for p, r in ((a, b), (a, c), (b, c))]
        if all(abs(x - 4.0) < 1e-9 for x in d):
            tris.append((a, b, c))
    return _unit(raw), sorted(tris)


def refine_sphere(x: np.ndarray, tris):
    """One 1:4 refinement of a spherical triangulation: the midpoint of every
    edge (edges sorted as ascending pairs) becomes a new vertex, numbered after
    the old ones in edge order and projected to the unit sphere."""
    edges = sorted({(min(p, r), max(p, r)) for t in tris
                    for p, r in ((t[0], t[1]), (t[0], t[2]), (t[1], t[2]))})
    eid = {e: len(x) + m for m, e in enumerate(edges)}
    mid = np.array([x[a] + x[b] for a, b in edges])
    xn = np.vstack([x, _unit(mid)])
    out = []
    for a, b, c in tris:
        ab, ac, bc = eid[(a, b)], eid[(a, c)], eid[(b, c)]
        for ch in ((a, ab, ac), (ab, b, bc), (ac, bc, c), (ab, bc, ac)):
            out.append(tuple(sorted(ch)))
    return xn, sorted(out)


@dataclass
class Shell:
    """Macro mesh T_{-2} of the shell with its primitive graph."""
    r1: float
    r2: float
    tang: int
    layers: int
    surf_x: np.ndarray = field(repr=False)      # (nS, 3) unit vectors
    tris: list = field(repr=False)              # surface triangles
    vert_x: np.ndarray = field(repr=False)      # (nV, 3) macro vertex positions
    vert_r: np.ndarray = field(repr=False)      # (nV,) radius of each vertex's layer
    vert_layer: np.ndarray = field(repr=False)  # (nV,)
    cells: np.ndarray = field(repr=False)       # (nC, 4) ascending ids
    edges: np.ndarray = field(repr=False)       # (nE, 2) sorted
    faces: np.ndarray = field(repr=False)       # (nF, 3) sorted
    edge_id: dict = field(repr=False)
    face_id: dict = field(repr=False)

    @property
    def nV(self):
        return len(self.vert_x)

    @property
    def nE(self):
        return len(self.edges)

    @property
    def nF(self):
        return len(self.faces)

    @property
    def nC(self):
        return len(self.cells)


def make_shell(r1: float = 0.55, r2: float = 1.0, tang: int = 0, layers: int = 1) -> Shell:
    """Icosahedral shell: surface refined `tang` times, `layers` radial layers
    at radii r1 + (r2 - r1) m / layers, each prism cut into three tetrahedra.

    For a surface triangle s0 < s1 < s2 with bottom vertices b and top vertices
    t the tetrahedra are {b0,b1,b2,t2}, {b0,b1,t1,t2}, {b0,t0,t1,t2}: every
    quadrilateral side is cut from the bottom of its lower id to the top of
    its higher id, so neighbouring prisms agree.  60 cells for (0, 1), 480 for
    (1, 2), 3840 for (2, 4), 30720 for (3, 8) (Sec. 4.1)."""
    xs, tris = icosahedron()
    for _ in range(tang):
        xs, tris = refine_sphere(xs, tris)
    nS = len(xs)
    M = layers
    radii = np.array([r1 + (r2 - r1) * m / M for m in range(M + 1)])
    vert_x = np.vstack([radii[m] * xs for m in range(M + 1)])
    vert_r = np.repeat(radii, nS)
    vert_layer = np.repeat(np.arange(M + 1), nS)
    cells = []
    for m in range(M):
        for s0, s1, s2 in tris:
            b0, b1, b2 = m * nS + s0, m * nS + s1, m * nS + s2
            t0, t1, t2 = b0 + nS, b1 + nS, b2 + nS
            cells.append((b0, b1, b2, t2))
            cells.append((b0, b1, t1, t2))
            cells.append((b0, t0, t1, t2))
    cells = np.array([sorted(c) for c in cells], dtype=np.int64)
    edges = sorted({(int(c[a]), int(c[b])) for c in cells
                    for a, b in itertools.combinations(range(4), 2)})
    faces = sorted({(int(c[a]), int(c[b]), int(c[d])) for c in cells
                    for a, b, d in itertools.combinations(range(4), 3)})
    return Shell(r1, r2, tang, layers, xs, tris, vert_x, vert_r, vert_layer, cells,
                 np.array(edges, dtype=np.int64), np.array(faces, dtype=np.int64),
                 {e: n for n, e in enumerate(edges)}, {f: n for n, f in enumerate(faces)})


# ----------------------------------------------------------------------------
# Index arithmetic on the refined macro cell
# ----------------------------------------------------------------------------

def n_face_nodes(N: int) -> int:
    return (N - 1) * (N - 2) // 2


def n_cell_nodes(N: int) -> int:
    """n_l of Eq. 2.5 with N = 2^(l+2)."""
    return (N - 1) * (N - 2) * (N - 3) // 6


def tet_count(n):
    """Points (a, b, c) >= 0 with a + b + c <= n."""
    return (n + 1) * (n + 2) * (n + 3) // 6


def lin_full(i, j, k, N):
    """Position of (i, j, k), i + j + k <= N, in the full macro cell with
    i fastest, then j, then k."""
    m = N - k
    return tet_count(N) - tet_count(N - k) + j * (m + 1) - j * (j - 1) // 2 + i


def lin_interior(i, j, k, N):
    """Position of an interior (i, j, k) among the n_l interior points."""
    return lin_full(i - 1, j - 1, k - 1, N - 4)


def lin_face(p, q, N):
    """Position of a face-interior point (p, q), p fastest."""
    return (q - 1) * (N - 1) - q * (q - 1) // 2 + (p - 1)


def full_points(N: int) -> np.ndarray:
    """All (i, j, k) with i + j + k <= N in lin_full order, shape (n, 3)."""
    pts = [(i, j, k) for k in range(N + 1) for j in range(N + 1 - k) for i in range(N + 1 - j - k)]
    return np.array(pts, dtype=np.int64)


def interior_points(N: int) -> np.ndarray:
    """The index triples I_l of Sec. 2.3 in lin_interior order, shape (n_l, 3)."""
    pts = [(i, j, k) for k in range(1, N) for j in range(1, N - k) for i in range(1, N - j - k)]
    return np.array(pts, dtype=np.int64).reshape(-1, 3)


# ----------------------------------------------------------------------------
# Level: the fine nodes of all primitives at N intervals per macro edge
# ----------------------------------------------------------------------------

@dataclass
class Level:
    shell: Shell
    N: int
    off_E: int
    off_F: int
    off_C: int
    n_total: int
    coords: np.ndarray = field(repr=False)     # (n_total, 3) mapped positions
    dirichlet: np.ndarray = field(repr=False)  # (n_total,) bool
    cell_map: np.ndarray = field(repr=False)   # (nC, n_full) canonical index of each cell-local point

    @property
    def free(self) -> np.ndarray:
        return np.flatnonzero(~self.dirichlet)


def _prim_offsets(sh: Shell, N: int):
    off_E = sh.nV
    off_F = off_E + sh.nE * (N - 1)
    off_C = off_F + sh.nF * n_face_nodes(N)
    n_total = off_C + sh.nC * n_cell_nodes(N)
    return off_E, off_F, off_C, n_total


def node_index(sh: Shell, N: int, gids: np.ndarray, lam: np.ndarray, cell: np.ndarray | None = None) -> np.ndarray:
    """Canonical index of the points with integer barycentric weights `lam`
    (rows sum to N) over the ascending global vertex ids `gids` (same shape).

    A point lies on the primitive spanned by the vertices with positive
    weight; its local index on that primitive is given by the weights of the
    primitive's second (and third) vertex.  Points with four positive weights
    are interior to `cell` (required then)."""
    off_E, off_F, off_C, _ = _prim_offsets(sh, N)
    gids = np.asarray(gids, dtype=np.int64)
    lam = np.asarray(lam, dtype=np.int64)
    out = np.full(len(lam), -1, dtype=np.int64)
    pos = lam > 0
    d = lam.shape[1]
    for pattern in itertools.product((False, True), repeat=d):
        if not any(pattern):
            continue
        sel = np.all(pos == np.array(pattern), axis=1)
        if not sel.any():
            continue
        cols = [a for a in range(d) if pattern[a]]
        g = gids[sel][:, cols]
        lm = lam[sel][:, cols]
        if len(cols) == 1:
            out[sel] = g[:, 0]
        elif len(cols) == 2:
            eids = np.array([sh.edge_id[(int(a), int(b))] for a, b in g], dtype=np.int64)
            out[sel] = off_E + eids * (N - 1) + (lm[:, 1] - 1)
        elif len(cols) == 3:
            fids = np.array([sh.face_id[(int(a), int(b), int(c))] for a, b, c in g], dtype=np.int64)
            out[sel] = off_F + fids * n_face_nodes(N) + lin_face(lm[:, 1], lm[:, 2], N)
        else:
            ijk = lm[:, 1:]
            out[sel] = off_C + cell[sel] * n_cell_nodes(N) + lin_interior(ijk[:, 0], ijk[:, 1], ijk[:, 2], N)
    return out


def blend(sh: Shell, gids: np.ndarray, lam: np.ndarray, N: int) -> np.ndarray:
    """Phi applied to the affine point sum_a lam_a v_a / N: the point is moved
    along its ray to radius rho = sum_a lam_a |v_a| / N (Sec. 2.2)."""
    lam = np.asarray(lam, dtype=np.float64)
    xh = np.zeros((len(lam), 3))
    rho = np.zeros(len(lam))
    for a in range(lam.shape[1]):
        xh = xh + lam[:, a:a + 1] * sh.vert_x[gids[:, a]]
        rho = rho + lam[:, a] * sh.vert_r[gids[:, a]]
    xh = xh / N
    rho = rho / N
    nrm = np.sqrt(xh[:, 0] * xh[:, 0] + xh[:, 1] * xh[:, 1] + xh[:, 2] * xh[:, 2])
    return rho[:, None] * xh / nrm[:, None]


def affine(sh: Shell, gids: np.ndarray, lam: np.ndarray, N: int) -> np.ndarray:
    """The unmapped point sum_a lam_a v_a / N (Phi = Id)."""
    lam = np.asarray(lam, dtype=np.float64)
    xh = np.zeros((len(lam), 3))
    for a in range(lam.shape[1]):
        xh = xh + lam[:, a:a + 1] * sh.vert_x[gids[:, a]]
    return xh / N


def cell_lambda(N: int, pts: np.ndarray) -> np.ndarray:
    """Barycentric weights (N - i - j - k, i, j, k) of cell-local points."""
    return np.column_stack([N - pts.sum(axis=1), pts[:, 0], pts[:, 1], pts[:, 2]])


def make_level(sh: Shell, N: int, mapped: bool = True) -> Level:
    """All fine nodes of level N: canonical positions (Phi applied unless
    mapped=False), Dirichlet mask and the per-cell local-to-canonical map."""
    assert N >= 4 and N & (N - 1) == 0
    off_E, off_F, off_C, n_total = _prim_offsets(sh, N)
    coords = np.zeros((n_total, 3))
    dirich = np.zeros(n_total, dtype=bool)
    place = blend if mapped else affine
    M = sh.layers
    lay = sh.vert_layer
    # vertices
    coords[:sh.nV] = sh.vert_x
    dirich[:sh.nV] = (lay == 0) | (lay == M)
    # edges
    p = np.arange(1, N)
    for e, (a, b) in enumerate(sh.edges):
        g = np.tile([a, b], (N - 1, 1))
        lam = np.column_stack([N - p, p])
        s = slice(off_E + e * (N - 1), off_E + (e + 1) * (N - 1))
        coords[s] = place(sh, g, lam, N)
        dirich[s] = (lay[a] == lay[b]) and lay[a] in (0, M)
    # faces
    fpts = np.array([(pp, qq) for qq in range(1, N - 1) for pp in range(1, N - qq)], dtype=np.int64).reshape(-1, 2)
    nf = n_face_nodes(N)
    for f, (a, b, c) in enumerate(sh.faces):
        g = np.tile([a, b, c], (nf, 1))
        lam = np.column_stack([N - fpts[:, 0] - fpts[:, 1], fpts[:, 0], fpts[:, 1]])
        s = slice(off_F + f * nf, off_F + (f + 1) * nf)
        if nf:
            coords[s] = place(sh, g, lam, N)
        dirich[s] = (lay[a] == lay[b] == lay[c]) and lay[a] in (0, M)
    # cells
    ipts = interior_points(N)
    nc = n_cell_nodes(N)
    lam_i = cell_lambda(N, ipts)
    for c in range(sh.nC):
        g = np.tile(sh.cells[c], (nc, 1))
        if nc:
            coords[off_C + c * nc: off_C + (c + 1) * nc] = place(sh, g, lam_i, N)
    # per-cell map of all local points
    fp = full_points(N)
    lam_f = cell_lambda(N, fp)
    nfull = len(fp)
    cmap = np.zeros((sh.nC, nfull), dtype=np.int64)
    for c in range(sh.nC):
        cmap[c] = node_index(sh, N, np.tile(sh.cells[c], (nfull, 1)), lam_f, np.full(nfull, c))
    return Level(sh, N, off_E, off_F, off_C, n_total, coords, dirich, cmap)


def support_kind(level: Level, idx: np.ndarray) -> np.ndarray:
    """0 vertex, 1 edge, 2 face, 3 cell interior for canonical indices."""
    idx = np.asarray(idx)
    return np.select([idx < level.off_E, idx < level.off_F, idx < level.off_C], [0, 1, 2], 3)


def offsets(sh: Shell, N: int):
    """(off_E, off_F, off_C, n_total) of the canonical order at level N."""
    return _prim_offsets(sh, N)


def dirichlet_of(sh: Shell, N: int, idx: np.ndarray) -> np.ndarray:
    """Dirichlet flag of canonical indices without building the level: a node
    is Dirichlet when its primitive's vertices all lie on r1 or all on r2."""
    off_E, off_F, off_C, _ = _prim_offsets(sh, N)
    idx = np.asarray(idx, dtype=np.int64)
    lay, M = sh.vert_layer, sh.layers
    out = np.zeros(len(idx), dtype=bool)
    v = idx < off_E
    out[v] = np.isin(lay[idx[v]], (0, M))
    e = (idx >= off_E) & (idx < off_F)
    if e.any():
        E = sh.edges[(idx[e] - off_E) // (N - 1)]
        la = lay[E]
        out[e] = (la[:, 0] == la[:, 1]) & np.isin(la[:, 0], (0, M))
    f = (idx >= off_F) & (idx < off_C)
    if f.any():
        F = sh.faces[(idx[f] - off_F) // n_face_nodes(N)]
        la = lay[F]
        out[f] = (la[:, 0] == la[:, 1]) & (la[:, 1] == la[:, 2]) & np.isin(la[:, 0], (0, M))
    return out


def primitive_of(sh: Shell, N: int, idx: int):
    """Vertex ids of the primitive that owns canonical node idx (1 to 4)."""
    off_E, off_F, off_C, _ = _prim_offsets(sh, N)
    if idx < off_E:
        return (int(idx),)
    if idx < off_F:
        return tuple(int(x) for x in sh.edges[(idx - off_E) // (N - 1)])
    if idx < off_C:
        return tuple(int(x) for x in sh.faces[(idx - off_F) // n_face_nodes(N)])
    return tuple(int(x) for x in sh.cells[(idx - off_C) // n_cell_nodes(N)])
