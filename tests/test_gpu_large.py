"""Full-size parity (3840 macro cells, N = 64, FP64: the benchmarked
workload) on sampled outputs the oracle computes one by one: interior rows of
seeded macro cells and seeded vertex / edge / face nodes, for apply, residual
and one smoother sweep (Eq. 5.1, 10 steps).  Bar: 1e-12 relative."""
import numpy as np
import pytest

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
    off_E, off_F, off_C, _ = M.offsets(sh, N)
    lower = np.concatenate([synthetic.sample(off_E, 3, 22), off_E + synthetic.sample(off_F - off_E, 6, 23),
                            off_F + synthetic.sample(off_C - off_F, 8, 24)])
    lower = lower[~M.dirichlet_of(sh, N, lower)]
    yield sh, s, u, f, cells, lower
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
    rows = LO.node_rows(sh, N, [int(x) for x in lower], opname)
    ref = np.array([sum(a * (0.0 if M.dirichlet_of(sh, N, [cc])[0] else u[cc]) for cc, a in rows[n].items())
                    for n in lower])
    assert rel(yh[lower], ref) <= TOL


def step_of(sh, idx):
    """Smoother step (0..9) of a free canonical node."""
    off_E, off_F, off_C, _ = M.offsets(sh, N)
    if idx < off_E:
        return 0
    if idx < off_F:
        p = (idx - off_E) % (N - 1) + 1
        return 1 + (p % 2)
    if idx < off_C:
        loc = (idx - off_F) % M.n_face_nodes(N)
        fp = [(pp, qq) for qq in range(1, N - 1) for pp in range(1, N - qq)]
        pp, qq = fp[loc]
        return 3 + (pp + 2 * qq) % 3
    ip = M.interior_points(N)[(idx - off_C) % M.n_cell_nodes(N)]
    return 6 + (ip[0] + 2 * ip[1] + 3 * ip[2]) % 4


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
    rows = LO.node_rows(sh, N, [int(x) for x in lower], opname)
    for n in lower:
        sn = step_of(sh, int(n))
        acc, diag = f[n], None
        for cc, a in rows[n].items():
            if cc == n:
                diag = a
                continue
            if M.dirichlet_of(sh, N, [cc])[0]:
                continue
            acc -= a * (ua[cc] if step_of(sh, cc) < sn else u[cc])
        assert abs(ua[n] - acc / diag) <= TOL * max(1.0, abs(acc / diag))
