"""Full-size FP32 parity of the staged surrogate smoother (one launch per sweep
for the four cell colours, planes staged in shared memory) on the
3840-macro shell at N = 64 and N = 128, the launch configurations the
benchmarks time.  One FP32 sweep (Eq. 5.1, 10 steps) is checked on sampled
outputs the FP64 oracle computes one by one from the same FP32-rounded
inputs: the interior rows of seeded macro cells (steps 7-10 from the state
the step order implies) and seeded vertex / edge / face nodes (steps 1-6).

FP32 bound: as in test_gpu_f32 -- each update is formed from O(15) FP32
terms, so the relative 2-norm error over a cell stays within a few hundred
FP32 ulps; the bar is 2e-5 relative."""
import numpy as np
import pytest

import synthetic
from oracle import local as LO
from oracle import mesh as M

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1608_06473_gb300 as hhg  # noqa: E402

TOL32 = 2e-5
TANG, LAYERS = 2, 4


@pytest.fixture(scope="module", params=[6, 7], ids=["N64", "N128"])
def big32(request):
    L = request.param
    N = 2 ** L
    sh = M.make_shell(tang=TANG, layers=LAYERS)
    s = hhg.Shell(0.55, 1.0, TANG, LAYERS, L)
    s.fit(2, 2)
    n_total, _ = s.num_nodes()
    u = synthetic.uniform(n_total, synthetic.SEED_U).astype(np.float32)
    f = synthetic.uniform(n_total, synthetic.SEED_F).astype(np.float32)
    cells = synthetic.sample(sh.nC, 3, 31)
    off_E, off_F, off_C, _ = M.offsets(sh, N)
    lower = np.concatenate([synthetic.sample(off_E, 3, 32), off_E + synthetic.sample(off_F - off_E, 6, 33),
                            off_F + synthetic.sample(off_C - off_F, 8, 34)])
    lower = lower[~M.dirichlet_of(sh, N, lower)]
    ut, ft = torch.from_numpy(u).cuda(), torch.from_numpy(f).cuda()
    s.smooth(ft, ut, 1, op=hhg.HHG_OP_LSQP, dtype=hhg.HHG_F32)
    torch.cuda.synchronize()
    ua = ut.cpu().numpy()
    del ut, ft
    torch.cuda.empty_cache()
    yield sh, N, u, f, ua, cells, lower
    s.close()


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def d(a, ix):
    """FP32 vector entries as FP64 (the oracle's arithmetic)."""
    return np.asarray(a[ix], dtype=np.float64)


def step_of(sh, N, idx):
    """Smoother step (0..9) of a free canonical node."""
    off_E, off_F, off_C, _ = M.offsets(sh, N)
    if idx < off_E:
        return 0
    if idx < off_F:
        p = (idx - off_E) % (N - 1) + 1
        return 1 + (p % 2)
    if idx < off_C:
        loc = (idx - off_F) % M.n_face_nodes(N)
        q = 1
        while loc >= N - 1 - q:
            loc -= N - 1 - q
            q += 1
        p = loc + 1
        return 3 + (p + 2 * q) % 3
    ip = M.interior_points(N)[(idx - off_C) % M.n_cell_nodes(N)]
    return 6 + (ip[0] + 2 * ip[1] + 3 * ip[2]) % 4


def test_f32_sweep_cell_interiors_sampled(big32):
    sh, N, u, f, ua, cells, _ = big32
    col = LO.colour_of(N)
    for c in cells:
        rows, cols, W = LO.interior_rows(sh, N, int(c), "lsqp")
        idx = np.unique(np.concatenate([rows, cols.ravel()]))
        start = np.where(np.isin(idx, rows), d(u, idx), d(ua, idx))
        start[M.dirichlet_of(sh, N, idx)] = 0.0
        lr, lc = np.searchsorted(idx, rows), np.searchsorted(idx, cols)
        got = LO.interior_colour_steps(lr, lc, W, col, start.copy(), d(f, idx))
        assert rel(d(ua, rows), got[lr]) <= TOL32


def test_f32_sweep_lower_primitives_sampled(big32):
    sh, N, u, f, ua, _, lower = big32
    rows = LO.node_rows(sh, N, [int(x) for x in lower], "lsqp")
    got, ref = [], []
    for n in lower:
        sn = step_of(sh, N, int(n))
        acc, diag = float(f[n]), None
        for cc, a in rows[n].items():
            if cc == n:
                diag = a
                continue
            if M.dirichlet_of(sh, N, [cc])[0]:
                continue
            acc -= a * float(ua[cc] if step_of(sh, N, cc) < sn else u[cc])
        got.append(float(ua[n]))
        ref.append(acc / diag)
    assert rel(np.array(got), np.array(ref)) <= TOL32
