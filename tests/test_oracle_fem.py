"""Pins of the oracle's exact operator L_l (element-wise P1 assembly on the
blended mesh, Sec. 2.2-2.3).  CPU only."""
import itertools

import numpy as np
import pytest

from oracle import fem as F
from oracle import mesh as M


def single_cell_shell(V):
    """A one-cell 'shell' with vertex positions V (4, 3) and no Dirichlet
    nodes, for closed-form checks with Phi = Id."""
    V = np.asarray(V, dtype=np.float64)
    edges = list(itertools.combinations(range(4), 2))
    faces = list(itertools.combinations(range(4), 3))
    return M.Shell(1.0, 2.0, 0, 2, None, [], V, np.linalg.norm(V, axis=1), np.ones(4, dtype=int),
                   np.array([[0, 1, 2, 3]]), np.array(edges), np.array(faces),
                   {e: n for n, e in enumerate(edges)}, {f: n for n, f in enumerate(faces)})


def test_kuhn_tets_count_and_cover():
    for N in (1, 2, 4, 8):
        t = F.kuhn_tets(N)
        assert len(t) == N ** 3                          # regular refinement: 8 children per level
        # affine reference tet (0, e1, e2, e3): volumes are all 1/(6 N^3)
        P = t.astype(float) / N
        E = P[:, 1:] - P[:, :1]
        vol = np.abs(np.linalg.det(E)) / 6
        assert np.allclose(vol, 1 / (6 * N ** 3), rtol=1e-12)
        assert np.isclose(vol.sum(), 1 / 6, rtol=1e-12)


def test_tets_per_node_and_edge_multiplicity():
    """24 tetrahedra meet at an interior node; of its 14 edges, 6 lie in 4
    tetrahedra and 8 in 6 (Sec. 4.2.1)."""
    N = 6
    t = F.kuhn_tets(N)
    x = np.array([2, 2, 1])
    around = [tt for tt in t if any((tt == x).all(axis=1))]
    assert len(around) == 24
    mult = []
    for w in F.DIRS[:14]:
        y = x + w
        mult.append(sum(1 for tt in around if any((tt == y).all(axis=1))))
    assert sorted(mult) == [4] * 6 + [6] * 8
    # the edge set of the refinement is exactly the 14 named directions
    E = {tuple(tt[b] - tt[a]) for tt in t for a in range(4) for b in range(4) if a != b}
    assert E == {tuple(w) for w in F.DIRS[:14]}


def test_element_stiffness_reference_tet():
    """Textbook: on (0, e1, e2, e3), grad(lambda) = (-1,-1,-1), e1, e2, e3 and
    |T| = 1/6."""
    P = np.array([[[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]]], dtype=float)
    K = F.element_stiffness(P)[0]
    ref = np.array([[3, -1, -1, -1], [-1, 1, 0, 0], [-1, 0, 1, 0], [-1, 0, 0, 1]]) / 6.0
    assert np.allclose(K, ref, rtol=0, atol=1e-15)
    # rigid motions leave K unchanged; scaling by s scales it by s (3-D)
    rng = np.random.default_rng(3)
    Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    P2 = 2.5 * P @ Q.T + rng.normal(size=3)
    assert np.allclose(F.element_stiffness(P2)[0], 2.5 * ref, rtol=1e-12, atol=1e-14)


@pytest.fixture(scope="module")
def c1_level8():
    sh = M.make_shell()
    lv = M.make_level(sh, 8)
    return lv, F.assemble(lv)


def test_symmetry_rowsum_patch(c1_level8):
    lv, A = c1_level8
    assert abs(A - A.T).max() < 1e-15                    # a_l is symmetric (Sec. 3.4)
    assert np.abs(np.asarray(A.sum(axis=1))).max() < 1e-14  # constants lie in V_l
    # linear patch test: (L x_d)_I = int grad phi_I . e_d = 0 at every node
    # not on the boundary (exact for P1 on straight tetrahedra)
    f = lv.free
    for d in range(3):
        assert np.abs((A @ lv.coords[:, d])[f]).max() < 1e-13


def test_stencil_has_15_points(c1_level8):
    lv, A = c1_level8
    rows = np.arange(lv.off_C, lv.n_total)
    nnz = np.diff(A.indptr)[rows]
    assert nnz.max() == 15


def test_constant_stencil_identity_map():
    """Phi = Id: all interior stencils of a macro cell are equal, opposite
    weights agree, and refining halves the stencil (s = 2^-l s_hat, Sec. 2.3)."""
    sh = M.make_shell()
    prev = None
    for N in (4, 8, 16):
        lv = M.make_level(sh, N, mapped=False)
        A = F.assemble(lv)
        S = F.interior_stencils(lv, A, cells=[0, 7, 33])
        assert np.abs(S - S[:, :1, :]).max() < 1e-14 * np.abs(S).max()
        s = S[:, 0, :]
        opp = {0: 1, 2: 3, 4: 5, 6: 10, 7: 11, 8: 12, 9: 13}
        for a, b in opp.items():
            assert np.allclose(s[:, a], s[:, b], rtol=0, atol=1e-14)
        if prev is not None:
            assert np.allclose(s, prev / 2, rtol=1e-12, atol=1e-15)
        prev = s


def test_freudenthal_cube_closed_form():
    """Cell (0, L e1, L(e1+e2), L(e1+e2+e3)) is a cubic lattice in
    (alpha, beta, gamma); its interior stencil is the 7-point Laplacian times h:
    mc = 6h, me = mw = mnw = mse = ts = bn = -h, the other 8 weights 0."""
    Lx = 1.7
    sh = single_cell_shell([[0, 0, 0], [Lx, 0, 0], [Lx, Lx, 0], [Lx, Lx, Lx]])
    N = 8
    h = Lx / N
    lv = M.make_level(sh, N, mapped=False)
    A = F.assemble(lv)
    S = F.interior_stencils(lv, A)[0]
    expect = np.zeros(15)
    expect[F.DIR_NAMES.index("mc")] = 6 * h
    for n in ("me", "mw", "mnw", "mse", "ts", "bn"):
        expect[F.DIR_NAMES.index(n)] = -h
    assert np.allclose(S, expect[None, :], rtol=0, atol=1e-14)


def test_volumes():
    """Phi = Id: the N^3 tetrahedra fill the polyhedral shell exactly; with Phi
    the volume tends to (4 pi / 3)(r2^3 - r1^3) at second order."""
    sh = M.make_shell()
    exact = 4 * np.pi / 3 * (1.0 - 0.55 ** 3)
    V = sh.vert_x[sh.cells]
    poly = np.abs(np.linalg.det(V[:, 1:] - V[:, :1])).sum() / 6
    loc = F.cell_tet_nodes(4)
    lv = M.make_level(sh, 4, mapped=False)
    P = lv.coords[lv.cell_map[:, loc]].reshape(-1, 4, 3)
    v4 = np.abs(np.linalg.det(P[:, 1:] - P[:, :1])).sum() / 6
    assert np.isclose(v4, poly, rtol=1e-13)
    errs = []
    for N in (4, 8, 16):
        lv = M.make_level(sh, N)
        loc = F.cell_tet_nodes(N)
        P = lv.coords[lv.cell_map[:, loc]].reshape(-1, 4, 3)
        errs.append(abs(np.abs(np.linalg.det(P[:, 1:] - P[:, :1])).sum() / 6 - exact))
    assert errs[0] > errs[1] > errs[2]
    assert errs[1] / errs[2] > 3.5
