"""Every launch configuration of the FP32 surrogate smoother (the
per-colour thread-per-node kernel with one or two nodes per thread in
flight, the shared-memory staged one-launch kernel at wavefront skew 1 and
2 with its CTA sizes, the plane-wavefront one-launch kernel with 128 and
256 threads, the per-colour kernel over line chunks, and the cell-resident
sweep with clusters of 1 (N <= 64) and 8 CTAs (N = 128)) against the FP64
oracle, on the 60-macro shell at N = 16 (whole vector) and N = 32 / 64
(sampled cells, the FP32 bound of test_gpu_f32: 2e-5 relative, and the
per-node bound of gpu_checks: C = 128 for two sweeps, 64 for one), pinned
through hhg_set_tuning; and the tuner's choice is a configuration that
fits."""
import numpy as np
import pytest

import gpu_checks as G
import synthetic
from oracle import fem as F
from oracle import local as LO
from oracle import lsqp as LS
from oracle import mesh as M
from oracle import mg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1608_06473_gb300 as hhg  # noqa: E402

TOL32 = 2e-5
CONFIGS = [-2, -1, 0, 1, 2, 3, 4, 5, 6, 7]


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def c1():
    sh = M.make_shell()
    lv = M.make_level(sh, 16)
    A = F.assemble(lv)
    B = LS.surrogate_operator(lv, A, LS.fit(lv, A, 2, 2), 2)
    s = hhg.Shell(0.55, 1.0, 0, 1, 4)
    s.fit(2, 2)
    yield lv, mg.Operator(lv, B), s
    s.close()


@pytest.mark.parametrize("cfg", CONFIGS)
def test_configs_whole_vector_n16(c1, cfg):
    lv, op, s = c1
    u = synthetic.uniform(lv.n_total, synthetic.SEED_U).astype(np.float32)
    f = synthetic.uniform(lv.n_total, synthetic.SEED_F).astype(np.float32)
    hhg.hhg_set_tuning(s.handle, 4, cfg)
    ut, ft = torch.from_numpy(u).cuda(), torch.from_numpy(f).cuda()
    s.smooth(ft, ut, 2, op=hhg.HHG_OP_LSQP, dtype=hhg.HHG_F32)
    torch.cuda.synchronize()
    ref = op.mask * u.astype(np.float64)
    for _ in range(2):
        ref = op.sweep(ref, f.astype(np.float64))
    got = ut.cpu().numpy().astype(np.float64)
    fr = lv.free
    assert rel(got[fr], ref[fr]) <= TOL32
    scale = (abs(op.off) @ np.abs(ref) + np.abs(f.astype(np.float64)))[fr] / np.abs(op.diag[fr])
    G.assert_per_node(got[fr], ref[fr], scale, 128, f"config {cfg}")


@pytest.mark.parametrize("L", [5, 6, 7])
def test_configs_sampled_cells(L):
    N = 2 ** L
    sh = M.make_shell()
    with hhg.Shell(0.55, 1.0, 0, 1, L) as s:
        s.fit(2, 2)
        n_total, _ = s.num_nodes()
        u = synthetic.uniform(n_total, synthetic.SEED_U).astype(np.float32)
        f = synthetic.uniform(n_total, synthetic.SEED_F).astype(np.float32)
        cells = synthetic.sample(sh.nC, 3, 41 + L)
        col = LO.colour_of(N)
        rows_of = {int(c): LO.interior_rows(sh, N, int(c), "lsqp") for c in cells}
        outs = {}
        for cfg in CONFIGS:
            hhg.hhg_set_tuning(s.handle, L, cfg)
            ut, ft = torch.from_numpy(u).cuda(), torch.from_numpy(f).cuda()
            s.smooth(ft, ut, 1, op=hhg.HHG_OP_LSQP, dtype=hhg.HHG_F32)
            torch.cuda.synchronize()
            ua = ut.cpu().numpy().astype(np.float64)
            outs[cfg] = ua
            for c, (rows, cols, W) in rows_of.items():
                idx = np.unique(np.concatenate([rows, cols.ravel()]))
                start = np.where(np.isin(idx, rows), u[idx].astype(np.float64), ua[idx])
                start[M.dirichlet_of(sh, N, idx)] = 0.0
                lr, lc = np.searchsorted(idx, rows), np.searchsorted(idx, cols)
                got = LO.interior_colour_steps(lr, lc, W, col, start.copy(), f[idx].astype(np.float64))
                assert rel(ua[rows], got[lr]) <= TOL32, (cfg, c)
                scale = G.cell_smoother_scale(W, lc, got, f[rows].astype(np.float64))
                G.assert_per_node(ua[rows], got[lr], scale, 64, f"config {cfg} cell {c}")
        # the configurations differ only in rounding order
        for cfg in CONFIGS:
            assert rel(outs[cfg], outs[-1]) <= TOL32


def test_tuner_choice_fits():
    with hhg.Shell(0.55, 1.0, 0, 1, 5) as s:
        s.fit(2, 2)
        n_total, _ = s.num_nodes()
        u = torch.zeros(n_total, dtype=torch.float32, device="cuda")
        s.smooth(u.clone(), u, 1, op=hhg.HHG_OP_LSQP, dtype=hhg.HHG_F32)
        torch.cuda.synchronize()
        for L in (3, 4, 5):
            cfg, ms = hhg.hhg_tuning(s.handle, L)
            assert cfg in CONFIGS
            assert ms[cfg + 2] > 0
            assert ms[cfg + 2] == min(m for m in ms if m > 0)
