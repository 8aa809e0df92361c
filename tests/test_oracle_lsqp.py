"""Pins of the oracle's least-squares surrogate (Sec. 3).  CPU only."""
import os

import numpy as np
import pytest

from oracle import fem as F
from oracle import local as LO
from oracle import lsqp as LS
from oracle import mesh as M

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_coefficient_counts():
    """m_q = (q+1)(q+2)(q+3)/6 (Eq. 3.2); 15 m_q L numbers per macro cell."""
    assert [LS.n_coeffs(q) for q in range(5)] == [1, 4, 10, 20, 35]
    for q in range(5):
        assert len(LS.monomials(q)) == LS.n_coeffs(q)
        assert len(set(LS.monomials(q))) == LS.n_coeffs(q)


def test_table43_sampling_counts():
    """|S_L| and sum_l |S_l| of Table 4.3 (L = 5) for S_l = M_{m(l, j)}."""
    rows = {l.split()[0]: (int(l.split()[1]), int(l.split()[2]))
            for l in open(os.path.join(GOLDEN, "table43_sampling_counts.txt"))
            if l.strip() and not l.startswith("#")}
    L = 5
    for name, jfun in (("LSQP_j2", lambda l: 2), ("LSQP_jlm1", lambda l: l - 1), ("LSQP_jl", lambda l: l)):
        sizes = [len(LS.sample_points(l, jfun(l))) for l in range(1, L + 1)]
        assert (sizes[-1], sum(sizes)) == rows[name]
    sizes = [len(LS.ipoly_points(4 * 2 ** l)) for l in range(1, L + 1)]
    assert (sizes[-1], sum(sizes)) == rows["IPOLY"]


@pytest.mark.parametrize("q", [1, 2, 3, 4])
def test_full_rank(q):
    """A has full rank for q <= 4 on every S_l = M_k, k >= 1 (Sec. 3.2)."""
    for l in (1, 2, 3):
        for k in range(1, l + 1):
            A = LS.design_matrix(LS.sample_points(l, k), 4 * 2 ** l, q)
            assert np.linalg.matrix_rank(A) == LS.n_coeffs(q)


@pytest.mark.parametrize("q", [1, 2, 3])
def test_exact_recovery_of_polynomial_weights(q):
    """Weights that already are polynomials of degree q are reproduced."""
    rng = np.random.default_rng(11 + q)
    N, l = 32, 3
    pts = LS.sample_points(l, 2)
    true = rng.normal(size=(14, LS.n_coeffs(q)))
    vals = LS.evaluate(true[None], pts, N, q)[0][:, :14]
    got = LS.fit_values(pts, N, q, vals)
    assert np.allclose(got, true, rtol=0, atol=1e-11 * np.abs(true).max())
    allp = M.interior_points(N)
    assert np.allclose(LS.evaluate(got[None], allp, N, q), LS.evaluate(true[None], allp, N, q),
                       rtol=0, atol=1e-12 * np.abs(true).max())


def test_affine_macro_gives_constant_exact_stencil():
    """Phi = Id: the surrogate reduces to the standard constant stencil (Sec. 3.4)."""
    sh = M.make_shell()
    N = 16
    lv = M.make_level(sh, N, mapped=False)
    A = F.assemble(lv)
    coef = LS.fit(lv, A, q=2, j=2, cells=[0, 21])
    ex = F.interior_stencils(lv, A, cells=[0, 21])
    su = LS.evaluate(coef, M.interior_points(N), N, 2)
    assert np.abs(su - ex).max() < 1e-13 * np.abs(ex).max()


def test_lemma_row_sum_of_fitted_polynomials():
    """Lemma of Sec. 3.4: fitting the centre weight too gives a_mc = -sum a_w."""
    sh = M.make_shell()
    N = 16
    pts = LS.sample_points(2, 2)
    for c in (3, 40):
        ex = LO.exact_stencils(sh, N, c, pts)
        coef = LS.fit_values(pts, N, 2, ex)            # all 15 columns
        assert np.abs(coef[14] + coef[:14].sum(axis=0)).max() < 1e-13 * np.abs(coef).max()


@pytest.mark.parametrize("q", [1, 2, 3])
def test_two_scale_decay(q):
    """Eq. 3.5 / Eq. 3.6: at fixed N the surrogate error falls like H^(q+1) under
    macro refinement 60 -> 480 -> 3840 (H halves each time).  Observed order
    in the finest pair must be at least q + 1 - 0.5."""
    rng = np.random.default_rng(5)
    N = 16
    ip = M.interior_points(N)
    pts = LS.sample_points(2, 2)
    worst = []
    for tang, layers in ((0, 1), (1, 2), (2, 4)):
        sh = M.make_shell(tang=tang, layers=layers)
        cells = rng.choice(sh.nC, 12, replace=False)
        w = 0.0
        for c in cells:
            ex = LO.exact_stencils(sh, N, c, ip)
            coef = LS.fit_values(pts, N, q, LO.exact_stencils(sh, N, c, pts)[:, :14])
            su = LS.evaluate(coef[None], ip, N, q)[0]
            _, einf = LS.fit_errors(ex[None], su[None])
            w = max(w, (einf[0, :14] / np.abs(ex[:, :14]).max()).max())
        worst.append(w)
    assert worst[0] > worst[1] > worst[2]
    assert np.log2(worst[1] / worst[2]) >= q + 1 - 0.5


def test_lsqp_beats_ipoly_in_l2_when_sampling_everything():
    """e_w^2 of LSQP on S = M_l is minimal over all quadratics, so it is <= the
    IPOLY value (Sec. 3.3); IPOLY interpolates at its ten points."""
    sh = M.make_shell()
    N = 16
    ip = M.interior_points(N)
    for c in (2, 31):
        ex = LO.exact_stencils(sh, N, c, ip)[:, :14]
        ls = LS.evaluate(LS.fit_values(ip, N, 2, ex)[None], ip, N, 2)[0][:, :14]
        p10 = LS.ipoly_points(N)
        ex10 = LO.exact_stencils(sh, N, c, p10)[:, :14]
        cip = LS.fit_values(p10, N, 2, ex10)
        assert np.allclose(LS.evaluate(cip[None], p10, N, 2)[0][:, :14], ex10, rtol=0, atol=1e-13)
        ipv = LS.evaluate(cip[None], ip, N, 2)[0][:, :14]
        e2_ls = np.sqrt(np.mean((ex - ls) ** 2, axis=0))
        e2_ip = np.sqrt(np.mean((ex - ipv) ** 2, axis=0))
        assert np.all(e2_ls <= e2_ip * (1 + 1e-12))


def test_surrogate_rows_sum_to_zero_and_lower_rows_exact():
    sh = M.make_shell()
    lv = M.make_level(sh, 8)
    A = F.assemble(lv)
    B = LS.surrogate_operator(lv, A, LS.fit(lv, A), 2)
    rs = np.asarray(B.sum(axis=1)).ravel()
    assert np.abs(rs).max() < 1e-14
    low = np.arange(lv.off_C)
    assert abs(B[low] - A[low]).max() == 0
    assert abs(B - A).max() > 0


def test_non_symmetry_is_first_order():
    """||L~^T - L~||_F / ||L||_F on one macro cell decays like h (Sec. 3.4)."""
    import scipy.sparse as sp
    sh = M.make_shell()
    c = 5
    out = []
    for N in (16, 32, 64):
        r, cols, W = LO.interior_rows(sh, N, c, "lsqp")
        _, _, We = LO.interior_rows(sh, N, c, "ifem")
        pos = np.full(cols.max() + 1, -1)
        pos[r] = np.arange(len(r))
        R, C, V, Ve = [], [], [], []
        for w in range(15):
            ok = pos[cols[:, w]] >= 0
            R.append(np.flatnonzero(ok))
            C.append(pos[cols[ok, w]])
            V.append(W[ok, w])
            Ve.append(We[ok, w])
        shp = (len(r), len(r))
        B = sp.coo_matrix((np.concatenate(V), (np.concatenate(R), np.concatenate(C))), shape=shp).tocsr()
        E = sp.coo_matrix((np.concatenate(Ve), (np.concatenate(R), np.concatenate(C))), shape=shp).tocsr()
        assert sp.linalg.norm(E - E.T) < 1e-14 * sp.linalg.norm(E)
        out.append(sp.linalg.norm(B - B.T) / sp.linalg.norm(E))
    assert out[0] > out[1] > out[2]
    assert 1.5 <= out[1] / out[2] <= 2.5


def test_ipoly_points_of_degree_q():
    """Sec. 3.1's points generalised to degree q: the m_q nodes of degree q of
    the shrunk cell (1,1,1), (N-3,1,1), (1,N-3,1), (1,1,N-3); q = 1 gives its
    vertices, q = 2 the ten listed points, q = 3 at N = 16 and 64 the exact
    lattice (1,1,1) + (N-4)/3 (a,b,c); elsewhere rounded, still distinct
    interior points with a nonsingular interpolation matrix."""
    for N in (8, 16, 32, 64, 128, 256):
        for q in (1, 2, 3):
            P = LS.ipoly_points(N, q)
            assert len(P) == LS.n_coeffs(q) == len({tuple(p) for p in P})
            assert np.all(P >= 1) and np.all(P.sum(axis=1) <= N - 1)
            assert np.linalg.matrix_rank(LS.design_matrix(P, N, q)) == LS.n_coeffs(q)
        v = {(1, 1, 1), (N - 3, 1, 1), (1, N - 3, 1), (1, 1, N - 3)}
        assert {tuple(p) for p in LS.ipoly_points(N, 1)} == v
        assert v <= {tuple(p) for p in LS.ipoly_points(N, 3)}
    for N in (16, 64):
        h = (N - 4) // 3
        lattice = {(1 + h * a, 1 + h * b, 1 + h * c) for a in range(4) for b in range(4 - a) for c in range(4 - a - b)}
        assert {tuple(p) for p in LS.ipoly_points(N, 3)} == lattice


@pytest.mark.parametrize("q", [1, 3])
def test_ipoly_of_degree_q_interpolates_and_recovers_polynomials(q):
    """IPOLY of degree q reproduces weights that are polynomials of degree q
    exactly, and interpolates the exact stencils at its points."""
    rng = np.random.default_rng(31 + q)
    N = 32
    P = LS.ipoly_points(N, q)
    true = rng.normal(size=(14, LS.n_coeffs(q)))
    vals = LS.evaluate(true[None], P, N, q)[0][:, :14]
    got = LS.fit_values(P, N, q, vals)
    allp = M.interior_points(N)
    assert np.allclose(LS.evaluate(got[None], allp, N, q), LS.evaluate(true[None], allp, N, q),
                       rtol=0, atol=1e-10 * np.abs(true).max())
    sh = M.make_shell()
    ex = LO.exact_stencils(sh, N, 5, P)[:, :14]
    cip = LS.fit_values(P, N, q, ex)
    assert np.allclose(LS.evaluate(cip[None], P, N, q)[0][:, :14], ex, rtol=0, atol=1e-12 * np.abs(ex).max())
