"""Pins of the oracle's smoother, transfers, coarse solve and V-cycle
(Sec. 4, Eq. 5.1).  CPU only."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import synthetic
from oracle import fem as F
from oracle import lsqp as LS
from oracle import mesh as M
from oracle import mg


@pytest.fixture(scope="module")
def c1_n8():
    sh = M.make_shell()
    lv = M.make_level(sh, 8)
    A = F.assemble(lv)
    B = LS.surrogate_operator(lv, A, LS.fit(lv, A), 2)
    return sh, lv, A, B


def test_colour_steps_partition_the_unknowns(c1_n8):
    sh, lv, A, _ = c1_n8
    steps = mg.colour_steps(lv)
    assert len(steps) == 10
    allidx = np.concatenate(steps)
    assert len(allidx) == len(np.unique(allidx))
    assert np.array_equal(np.sort(allidx), lv.free)


def test_cell_and_face_steps_are_independent_sets(c1_n8):
    """No two nodes of one cell step are coupled (a proper colouring, Sec. 5);
    within one face the three face colours are proper too."""
    sh, lv, A, _ = c1_n8
    S = (A != 0).astype(np.float64)
    steps = mg.colour_steps(lv)
    for s in steps[6:]:
        blk = S[s][:, s]
        assert (blk - sp.diags(blk.diagonal())).nnz == 0
    nf = M.n_face_nodes(lv.N)
    for s in steps[3:6]:
        face = (s - lv.off_F) // nf
        blk = S[s][:, s].tocoo()
        off = blk.row != blk.col
        assert np.all(face[blk.row[off]] != face[blk.col[off]])


def test_sweep_matches_pointwise_formula(c1_n8):
    """Each step applies Eq. 5.1 to every node of its set with the values at
    the start of the step; checked row by row against the matrix entries."""
    sh, lv, A, B = c1_n8
    op = mg.Operator(lv, B)
    f = synthetic.uniform(lv.n_total, 0)
    u = op.mask * synthetic.uniform(lv.n_total, 1)
    got = op.sweep(u, f)
    ref = u.copy()
    Bc = B.tocsr()
    for S in op.steps:
        old = ref.copy()
        for I in S:
            lo, hi = Bc.indptr[I], Bc.indptr[I + 1]
            acc, diag = f[I], None
            for J, a in zip(Bc.indices[lo:hi], Bc.data[lo:hi]):
                if J == I:
                    diag = a
                else:
                    acc -= a * old[J]
            ref[I] = acc / diag
    assert np.allclose(got, ref, rtol=0, atol=1e-13 * np.abs(ref).max())


def test_prolongation_reproduces_linear_functions():
    """Phi = Id: every new fine node is the midpoint of a coarse edge, so P
    maps the coarse coordinate functions to the fine ones and constants to
    constants."""
    sh = M.make_shell()
    for N in (8, 16):
        lf = M.make_level(sh, N, mapped=False)
        lc = M.make_level(sh, N // 2, mapped=False)
        P = mg.prolongation(lf, lc)
        assert np.allclose(P @ np.ones(lc.n_total), 1.0, rtol=0, atol=1e-15)
        for d in range(3):
            assert np.allclose(P @ lc.coords[:, d], lf.coords[:, d], rtol=0, atol=1e-15)


def test_galerkin_identity_for_nested_affine_meshes():
    """Phi = Id: the meshes are nested, V_{l-1} is a subspace of V_l and
    P^T L_l P = L_{l-1} exactly."""
    sh = M.make_shell()
    lf = M.make_level(sh, 8, mapped=False)
    lc = M.make_level(sh, 4, mapped=False)
    P = mg.prolongation(lf, lc)
    G = (P.T @ F.assemble(lf) @ P).tocsr()
    Ac = F.assemble(lc)
    assert abs(G - Ac).max() < 1e-14 * abs(Ac).max()


def test_restriction_is_the_transpose(c1_n8):
    sh, lv, A, _ = c1_n8
    lc = M.make_level(sh, 4)
    tr = mg.Transfer(lv, lc)
    r = synthetic.uniform(lv.n_total, 3)
    e = synthetic.uniform(lc.n_total, 4)
    assert np.isclose(tr.restrict(r) @ e, r @ tr.prolong(e), rtol=1e-13)
    assert np.all(tr.prolong(e)[lv.dirichlet] == 0)
    assert np.all(tr.restrict(r)[lc.dirichlet] == 0)


def test_sweeps_reduce_the_energy_error():
    """Exact L is SPD on the unknowns: smoothing reduces the energy norm of the
    error, sweep after sweep."""
    sh = M.make_shell()
    lv = M.make_level(sh, 8)
    op = mg.Operator(lv, F.assemble(lv))
    fr = lv.free
    f = op.mask * synthetic.uniform(lv.n_total, 0)
    Aff = op.A[fr][:, fr]
    x = np.zeros(lv.n_total)
    x[fr] = spla.spsolve(Aff.tocsc(), f[fr])
    u = op.mask * synthetic.uniform(lv.n_total, 1)
    prev = np.inf
    for _ in range(6):
        u = op.sweep(u, f)
        e = (u - x)[fr]
        en = e @ (Aff @ e)
        assert en < prev
        prev = en


def test_coarse_solve_is_exact():
    sh = M.make_shell()
    lv = M.make_level(sh, 4)
    op = mg.Operator(lv, F.assemble(lv))
    cs = mg.CoarseSolver(op)
    f = synthetic.uniform(lv.n_total, 0)
    u = cs.solve(op.mask * f)
    assert np.linalg.norm(op.residual(u, f)) <= 1e-13 * np.linalg.norm(op.mask * f)


@pytest.mark.parametrize("opname", ["lsqp", "ifem"])
def test_vcycle_converges_to_the_discrete_solution(opname):
    sh = M.make_shell()
    H = mg.build_hierarchy(sh, 16, opname)
    lv = H.levels[-1]
    f = synthetic.uniform(lv.n_total, synthetic.SEED_F)
    u, hist = H.solve(f, rtol=1e-8, max_cycles=20)
    assert hist[-1] <= 1e-8 and len(hist) <= 15
    rates = np.array(hist[1:]) / np.array(hist[:-1])
    assert rates[2:].max() < 0.3
    fr = lv.free
    A = H.ops[-1].A[fr][:, fr]
    x = spla.spsolve(A.tocsc(), f[fr])
    assert np.linalg.norm(u[fr] - x) <= 1e-6 * np.linalg.norm(x)


def test_dd_with_equal_operators_is_the_plain_cycle():
    """Double discretisation reduces to the standard V-cycle when the
    relaxation and residual operators coincide."""
    sh = M.make_shell()
    H = mg.build_hierarchy(sh, 16, "lsqp")
    Hd = mg.Hierarchy(H.levels, H.ops, list(H.ops))
    f = synthetic.uniform(H.levels[-1].n_total, synthetic.SEED_F)
    u = np.zeros_like(f)
    a = H.vcycle(len(H.ops) - 1, u, f)
    b = Hd.vcycle(len(Hd.ops) - 1, u, f)
    assert np.array_equal(a, b)


def test_cons_dd_on_the_unprojected_domain_is_the_plain_cycle():
    """CONS DD relaxes with the stencils of the unprojected domain in the cell
    interiors; on an unprojected shell those are the exact operator's own
    rows, so its relaxation operator equals the exact one and the cycle is the
    plain FEM cycle (to the rounding of re-reading the rows)."""
    sh = M.make_shell()
    Hc = mg.build_hierarchy(sh, 16, "dd-cons", mapped=False)
    He = mg.build_hierarchy(sh, 16, "ifem", mapped=False)
    for a, b in zip(Hc.smooth_ops, He.ops):
        assert abs(a.A - b.A).max() <= 1e-14 * abs(b.A).max()
    f = synthetic.uniform(He.levels[-1].n_total, synthetic.SEED_F)
    u = np.zeros_like(f)
    x = Hc.vcycle(len(Hc.ops) - 1, u, f)
    y = He.vcycle(len(He.ops) - 1, u, f)
    assert np.linalg.norm(x - y) <= 1e-12 * np.linalg.norm(y)


def test_dd_recovers_the_exact_operator_solution():
    """Sec. 4.1: relaxing with the surrogate and computing residuals with the
    exact operator moves the iterate towards the exact operator's solution
    L^-1 f: closer to it than the surrogate's own solution L~^-1 f, for both
    LSQP and IPOLY (on this random right-hand side by a factor of about 0.6;
    the bar is 0.75); the update norms fall to the stopping tolerance."""
    sh = M.make_shell()
    Hx = mg.build_hierarchy(sh, 16, "ifem")
    lv = Hx.levels[-1]
    fr = lv.free
    f = synthetic.uniform(lv.n_total, synthetic.SEED_F)
    x = spla.spsolve(Hx.ops[-1].A[fr][:, fr].tocsc(), f[fr])
    for kind in ("lsqp", "ipoly"):
        Hs = mg.build_hierarchy(sh, 16, kind)
        xs = spla.spsolve(Hs.ops[-1].A[fr][:, fr].tocsc(), f[fr])
        Hd = mg.build_hierarchy(sh, 16, "dd-" + kind)
        u, hist = Hd.solve_updates(f, rtol=1e-8, max_cycles=40)
        assert hist[-1] <= 1e-8
        assert np.linalg.norm(u[fr] - x) < 0.75 * np.linalg.norm(xs - x)


def test_ipoly_hierarchy_converges():
    sh = M.make_shell()
    H = mg.build_hierarchy(sh, 16, "ipoly")
    f = synthetic.uniform(H.levels[-1].n_total, synthetic.SEED_F)
    _, hist = H.solve(f, rtol=1e-8, max_cycles=20)
    assert hist[-1] <= 1e-8
