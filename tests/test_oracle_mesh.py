"""Pins of the oracle's macro mesh, blending map and canonical node order
(Sec. 2.2-2.3).  CPU only."""
import numpy as np
import pytest

from oracle import mesh as M


@pytest.mark.parametrize("tang,layers,nc", [(0, 1, 60), (1, 2, 480), (2, 4, 3840)])
def test_macro_counts_and_euler(tang, layers, nc):
    sh = M.make_shell(tang=tang, layers=layers)
    assert sh.nC == nc                      # Sec. 4.1: 60 / 480 / 3840 macro cells
    # the shell is a ball with a hole: V - E + F - C = 2 for its tetrahedral complex
    assert sh.nV - sh.nE + sh.nF - sh.nC == 2
    # every face is shared by at most two cells; boundary faces lie on r1 or r2
    cnt = {}
    for c in sh.cells:
        for f in ((c[0], c[1], c[2]), (c[0], c[1], c[3]), (c[0], c[2], c[3]), (c[1], c[2], c[3])):
            cnt[tuple(int(x) for x in f)] = cnt.get(tuple(int(x) for x in f), 0) + 1
    assert max(cnt.values()) == 2
    for f, n in cnt.items():
        if n == 1:
            lay = {int(sh.vert_layer[v]) for v in f}
            assert lay in ({0}, {layers})


def test_c1_counts():
    sh = M.make_shell()
    assert (sh.nV, sh.nE, sh.nF, sh.nC) == (24, 102, 140, 60)
    lv = M.make_level(sh, 16)
    # (N_r + 1) radial node layers of 10 n_t^2 + 2 surface nodes
    assert lv.n_total == 17 * (10 * 16 ** 2 + 2) == 43554
    assert (~lv.dirichlet).sum() == 43554 - 2 * 2562 == 38430


@pytest.mark.parametrize("tang,layers,N,total", [(2, 4, 64, 168428034), (2, 4, 128, 1344799746),
                                                 (2, 4, 32, 21135618)])
def test_large_shell_node_totals(tang, layers, N, total):
    sh = M.make_shell(tang=tang, layers=layers)
    nt = N * 2 ** tang
    assert M._prim_offsets(sh, N)[3] == (N * layers + 1) * (10 * nt ** 2 + 2) == total


def test_vertex_radii_and_blending():
    sh = M.make_shell(r1=0.55, r2=1.0, tang=1, layers=2)
    r = np.linalg.norm(sh.vert_x, axis=1)
    assert np.allclose(r, sh.vert_r, rtol=0, atol=1e-15)
    assert set(np.round(sh.vert_r, 12)) == {0.55, 0.775, 1.0}
    lv = M.make_level(sh, 8)
    # Phi fixes the macro vertices
    assert np.array_equal(lv.coords[:sh.nV], sh.vert_x)
    # nodes on the two boundary spheres are mapped onto them (to rounding)
    rad = np.linalg.norm(lv.coords[lv.dirichlet], axis=1)
    on_in = np.isclose(rad, 0.55, rtol=0, atol=1e-14)
    on_out = np.isclose(rad, 1.0, rtol=0, atol=1e-14)
    assert np.all(on_in | on_out)
    # every mapped node of an interior radial layer lies on that layer's sphere
    # when it is on a face whose vertices share the layer
    for f, (a, b, c) in enumerate(sh.faces):
        if sh.vert_layer[a] == sh.vert_layer[b] == sh.vert_layer[c]:
            nf = M.n_face_nodes(8)
            x = lv.coords[lv.off_F + f * nf: lv.off_F + (f + 1) * nf]
            assert np.allclose(np.linalg.norm(x, axis=1), sh.vert_r[a], rtol=0, atol=1e-14)


def test_cell_local_positions_agree_across_cells():
    """Phi is continuous: the position of a shared node computed from every
    adjacent cell's local formula equals its canonical position exactly
    (macro vertices, whose canonical position is the vertex itself, to an
    ulp)."""
    sh = M.make_shell()
    N = 8
    lv = M.make_level(sh, N)
    fp = M.full_points(N)
    lam = M.cell_lambda(N, fp)
    for c in range(sh.nC):
        x = M.blend(sh, np.tile(sh.cells[c], (len(fp), 1)), lam, N)
        y = lv.coords[lv.cell_map[c]]
        vert = lv.cell_map[c] < sh.nV
        assert np.array_equal(x[~vert], y[~vert])
        assert np.allclose(x[vert], y[vert], rtol=0, atol=2e-16)


def test_canonical_order_is_a_bijection():
    sh = M.make_shell()
    N = 8
    lv = M.make_level(sh, N)
    seen = np.zeros(lv.n_total, dtype=int)
    for c in range(sh.nC):
        seen[np.unique(lv.cell_map[c])] += 1
    assert seen.min() >= 1                      # every node lies in some cell
    nc = M.n_cell_nodes(N)
    assert np.all(seen[lv.off_C:] == 1)         # interior nodes in exactly one cell
    # interior block of cell c is contiguous in lin_interior order
    ip = M.interior_points(N)
    for c in (0, 17, 59):
        idx = lv.cell_map[c][M.lin_full(ip[:, 0], ip[:, 1], ip[:, 2], N)]
        assert np.array_equal(idx, lv.off_C + c * nc + np.arange(nc))


def test_index_formulas():
    for N in (4, 8, 16):
        fp = M.full_points(N)
        assert np.array_equal(M.lin_full(fp[:, 0], fp[:, 1], fp[:, 2], N), np.arange(len(fp)))
        ip = M.interior_points(N)
        assert np.array_equal(M.lin_interior(ip[:, 0], ip[:, 1], ip[:, 2], N), np.arange(len(ip)))
        fpts = [(p, q) for q in range(1, N - 1) for p in range(1, N - q)]
        assert [M.lin_face(p, q, N) for p, q in fpts] == list(range(len(fpts)))


def test_interior_counts_golden():
    rows = [l.split() for l in open(__file__.replace("test_oracle_mesh.py", "golden/interior_counts.txt"))
            if l.strip() and not l.startswith("#")]
    for l, n in rows:
        N = 2 ** (int(l) + 2)
        assert M.n_cell_nodes(N) == int(n)
        if N <= 64:
            assert len(M.interior_points(N)) == int(n)
