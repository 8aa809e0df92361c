"""Reduced precision: FP32 operator application, residual and smoother
against the FP64 oracle (on the same FP32-rounded inputs), and the
mixed-precision solve (FP32 V-cycles inside FP64 iterative refinement)
against the FP64 solve.

FP32 bound: every weight and every update is formed from O(15) FP32 terms
whose magnitudes exceed the result by the row's cancellation factor (about
4 for random u), so the relative 2-norm error stays within a few hundred
FP32 ulps; the bar used is 2e-5 (= 168 eps_32) relative.  Every node must
also meet the per-node bound of gpu_checks (C = 64 for apply, residual and
one sweep, 128 for two sweeps), so no wrong node hides in the norm."""
import numpy as np
import pytest

import gpu_checks as G
import synthetic
from oracle import fem as F
from oracle import lsqp as LS
from oracle import mesh as M
from oracle import mg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1608_06473_gb300 as hhg  # noqa: E402

TOL32 = 2e-5
OPS = {"ifem": hhg.HHG_OP_IFEM, "lsqp": hhg.HHG_OP_LSQP}


@pytest.fixture(scope="module")
def c1():
    sh = M.make_shell()
    lv = M.make_level(sh, 16)
    A = F.assemble(lv)
    B = LS.surrogate_operator(lv, A, LS.fit(lv, A, 2, 2), 2)
    s = hhg.Shell(0.55, 1.0, 0, 1, 4)
    s.fit(2, 2)
    yield lv, {"ifem": mg.Operator(lv, A), "lsqp": mg.Operator(lv, B)}, s
    s.close()


def rel(a, b, free):
    return np.linalg.norm(a[free] - b[free]) / np.linalg.norm(b[free])


def f32(x):
    return np.asarray(x, dtype=np.float32)


@pytest.mark.parametrize("opname", ["ifem", "lsqp"])
def test_f32_apply_residual(c1, opname):
    lv, ops, s = c1
    u = f32(synthetic.uniform(lv.n_total, synthetic.SEED_U))
    f = f32(synthetic.uniform(lv.n_total, synthetic.SEED_F))
    ut, ft = torch.from_numpy(u).cuda(), torch.from_numpy(f).cuda()
    y, r = torch.empty_like(ut), torch.empty_like(ut)
    s.apply(ut, y, op=OPS[opname], dtype=hhg.HHG_F32)
    nrm = s.residual(ut, ft, r, op=OPS[opname], dtype=hhg.HHG_F32)[0]
    torch.cuda.synchronize()
    op = ops[opname]
    yr = op.apply(u.astype(np.float64))
    rr = op.residual(u.astype(np.float64), f.astype(np.float64))
    yg, rg = y.cpu().numpy().astype(np.float64), r.cpu().numpy().astype(np.float64)
    assert rel(yg, yr, lv.free) <= TOL32
    assert rel(rg, rr, lv.free) <= TOL32
    absAu = abs(op.A) @ np.abs(op.mask * u.astype(np.float64))
    fr = lv.free
    G.assert_per_node(yg[fr], yr[fr], absAu[fr], 64, "apply")
    G.assert_per_node(rg[fr], rr[fr], absAu[fr] + np.abs(f[fr].astype(np.float64)), 64, "residual")
    assert abs(nrm - np.linalg.norm(rr)) <= TOL32 * np.linalg.norm(rr)


@pytest.mark.parametrize("opname", ["ifem", "lsqp"])
def test_f32_smoother(c1, opname):
    lv, ops, s = c1
    u = f32(synthetic.uniform(lv.n_total, synthetic.SEED_U))
    f = f32(synthetic.uniform(lv.n_total, synthetic.SEED_F))
    ut, ft = torch.from_numpy(u).cuda(), torch.from_numpy(f).cuda()
    s.smooth(ft, ut, 2, op=OPS[opname], dtype=hhg.HHG_F32)
    torch.cuda.synchronize()
    op = ops[opname]
    ref = op.mask * u.astype(np.float64)
    for _ in range(2):
        ref = op.sweep(ref, f.astype(np.float64))
    got = ut.cpu().numpy().astype(np.float64)
    assert rel(got, ref, lv.free) <= TOL32
    fr = lv.free
    scale = (abs(op.off) @ np.abs(ref) + np.abs(f.astype(np.float64)))[fr] / np.abs(op.diag[fr])
    G.assert_per_node(got[fr], ref[fr], scale, 128, "two sweeps")


@pytest.mark.parametrize("opname", ["ifem", "lsqp"])
def test_mixed_precision_solve(c1, opname):
    """FP32 inner cycles, FP64 refinement: reaches the FP64 tolerance on the
    FP64 residual and the same solution as the FP64 solve."""
    lv, ops, s = c1
    f = synthetic.uniform(lv.n_total, synthetic.SEED_F)
    ft = torch.from_numpy(f).cuda()
    u64 = torch.zeros_like(ft)
    rel64, cyc64, _ = s.vcycle(ft, u64, op=OPS[opname], dtype=hhg.HHG_F64, rtol=1e-8)
    u32 = torch.zeros_like(ft)
    rel32, cyc32, _ = s.vcycle(ft, u32, op=OPS[opname], dtype=hhg.HHG_F32, rtol=1e-8)
    assert rel32[0] <= 1e-8
    assert cyc32 <= cyc64 + 3
    r = torch.empty_like(ft)
    nrm = s.residual(u32, ft, r, op=OPS[opname])[0]
    r0 = np.linalg.norm(ops[opname].residual(np.zeros(lv.n_total), f))
    assert nrm <= 1e-8 * r0 * (1 + 1e-6)
    a, b = u32.cpu().numpy(), u64.cpu().numpy()
    assert rel(a, b, lv.free) <= 1e-6
