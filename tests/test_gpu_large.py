"""Full-size parity (3840 macro cells, N = 64, FP64: the benchmarked
workload) on sampled outputs the oracle computes one by one: interior rows of
seeded macro cells and seeded vertex / edge / face nodes, for apply, residual
and one smoother sweep (Eq. 5.1, 10 steps).  Bar: 1e-12 relative.  Lower
nodes: a few hundred on the boundaries of two seeded cells (their rows are
exact in both operators, so one oracle assembly serves both)."""
import numpy as np
import pytest

import gpu_checks as G
import synthetic
from oracle import local as LO
from oracle import mesh as M

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1608_06473_gb300 as hhg  # noqa: E402

TANG, LAYERS, L = 2, 4, 6
N = 2 ** L
TOL = 1e-12


@pytest.fixture(scope="module")
def big():
    sh = M.make_shell(tang=TANG, layers=LAYERS)
    s = hhg.Shell(0.55, 1.0, TANG, LAYERS, L)
    s.fit(2, 2)
    n_total, _ = s.num_nodes()
    u = synthetic.uniform(n_total, synthetic.SEED_U)
    f = synthetic.uniform(n_total, synthetic.SEED_F)
    cells = synthetic.sample(sh.nC, 4, 21)
    lower = G.lower_sample(sh, N, cells[:2], 150, 22)
    rows = LO.node_rows(sh, N, [int(x) for x in lower], "ifem")
    yield sh, s, u, f, cells, (lower, rows)
    s.close()


def masked(sh, u, cols):
    return np.where(M.dirichlet_of(sh, N, cols.ravel()).reshape(cols.shape), 0.0, u[cols])


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("opname", ["lsqp", "ifem"])
def test_apply_and_residual_sampled(big, opname):
    sh, s, u, f, cells, lower = big
    op = hhg.HHG_OP_LSQP if opname == "lsqp" else hhg.HHG_OP_IFEM
    ut, ft = torch.from_numpy(u).cuda(), torch.from_numpy(f).cuda()
    y = torch.empty_like(ut)
    r = torch.empty_like(ut)
    s.apply(ut, y, op=op)
    nrm = s.residual(ut, ft, r, op=op)[0]
    torch.cuda.synchronize()
    yh, rh = y.cpu().numpy(), r.cpu().numpy()
    assert np.isclose(nrm, np.linalg.norm(rh), rtol=1e-13)
    for c in cells:
        rows, cols, W = LO.interior_rows(sh, N, int(c), opname)
        ref = (W * masked(sh, u, cols)).sum(axis=1)
        assert rel(yh[rows], ref) <= TOL
        assert rel(rh[rows], f[rows] - ref) <= TOL
    lower, rows = lower
    assert len(lower) >= 150
    ref = np.array([sum(a * (0.0 if M.dirichlet_of(sh, N, [cc])[0] else u[cc]) for cc, a in rows[n].items())
                    for n in lower])
    assert rel(yh[lower], ref) <= TOL
    assert rel(rh[lower], f[lower] - ref) <= TOL


@pytest.mark.parametrize("opname", ["lsqp", "ifem"])
def test_one_sweep_sampled(big, opname):
    """u_after of one GPU sweep against Eq. 5.1 per sampled node, with each
    neighbour taken at the state its step order implies (updated earlier in
    the sweep -> u_after, later -> u_before)."""
    sh, s, u, f, cells, lower = big
    op = hhg.HHG_OP_LSQP if opname == "lsqp" else hhg.HHG_OP_IFEM
    ut, ft = torch.from_numpy(u).cuda(), torch.from_numpy(f).cuda()
    s.smooth(ft, ut, 1, op=op)
    torch.cuda.synchronize()
    ua = ut.cpu().numpy()
    # cell interiors: steps 7-10 start from u_before inside, u_after on the cell boundary
    col = LO.colour_of(N)
    for c in cells:
        rows, cols, W = LO.interior_rows(sh, N, int(c), opname)
        idx = np.unique(np.concatenate([rows, cols.ravel()]))
        start = np.where(np.isin(idx, rows), u[idx], ua[idx])
        start[M.dirichlet_of(sh, N, idx)] = 0.0
        lr, lc = np.searchsorted(idx, rows), np.searchsorted(idx, cols)
        got = LO.interior_colour_steps(lr, lc, W, col, start.copy(), f[idx])
        assert rel(ua[rows], got[lr]) <= TOL
    # lower primitives: steps 1-6
    lower, rows = lower
    ref, scale = G.lower_sweep_reference(sh, N, rows, lower, u, ua, f)
    assert rel(ua[lower], ref) <= TOL
    # per node, against the magnitude of the terms of Eq. 5.1 (an update
    # may cancel to far below its terms)
    assert np.all(np.abs(ua[lower] - ref) <= TOL * scale)
