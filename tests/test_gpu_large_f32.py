"""Full-size FP32 parity of the staged surrogate smoother (one launch per sweep
for the four cell colours, planes staged in shared memory) on the
3840-macro shell at N = 64 and N = 128, the launch configurations the
benchmarks time.  One FP32 sweep (Eq. 5.1, 10 steps) is checked on sampled
outputs the FP64 oracle computes one by one from the same FP32-rounded
inputs: the interior rows of seeded macro cells (steps 7-10 from the state
the step order implies) and seeded vertex / edge / face nodes (steps 1-6).

FP32 bounds: as in test_gpu_f32 -- each update is formed from O(15) FP32
terms, so the relative 2-norm error over a cell stays within a few hundred
FP32 ulps; the bar is 2e-5 relative.  Every sampled node must also meet the
per-node bound of gpu_checks (C = 64 for one sweep): a few wrong nodes next
to a cell boundary cannot hide in the norm.  Lower nodes: a few hundred on
the boundaries of seeded cells."""
import numpy as np
import pytest

import gpu_checks as G
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
    # a few hundred lower nodes around one or two cells (the oracle assembles
    # every cell that holds a sampled node)
    if N == 64:
        lower = G.lower_sample(sh, N, cells[:2], 150, 32)
    else:
        lower = G.lower_sample(sh, N, cells[:1], 200, 32, vertices=False)
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
        scale = G.cell_smoother_scale(W, lc, got, d(f, rows))
        G.assert_per_node(d(ua, rows), got[lr], scale, 64, f"cell {c}")


def test_f32_sweep_lower_primitives_sampled(big32):
    sh, N, u, f, ua, _, lower = big32
    assert len(lower) >= 150
    rows = LO.node_rows(sh, N, [int(x) for x in lower], "ifem")
    ref, scale = G.lower_sweep_reference(sh, N, rows, lower, u, ua, f)
    got = d(ua, lower)
    assert rel(got, ref) <= TOL32
    G.assert_per_node(got, ref, scale, 64, "lower nodes")
