"""LSQP surrogates of degree q = 1 and 3 and sampling sets j = 1 and 3
(Sec. 3.2, S_l = M_{m(l,j)}), and IPOLY of degree 1 and 3 (Sec. 3.1), on the
GPU against the FP64 oracle: FP64 apply and one smoother sweep to 1e-12
relative, FP32 apply to 2e-5 relative (the FP32 bar of the q = 2 tests), on
the 60-cell shell at N = 8 and 16, and at N = 32 for j = 3 (the first level
where m(l, 3) differs from m(l, 2))."""
import numpy as np
import pytest

import synthetic
from oracle import fem as F
from oracle import lsqp as LS
from oracle import mesh as M
from oracle import mg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1608_06473_gb300 as hhg  # noqa: E402

TOL32 = 2e-5


def rel(a, b, free):
    return np.linalg.norm(a[free] - b[free]) / np.linalg.norm(b[free])


@pytest.fixture(scope="module")
def setup():
    sh = M.make_shell()
    levels = {l2: M.make_level(sh, 2 ** l2) for l2 in (3, 4, 5)}
    As = {l2: F.assemble(lv) for l2, lv in levels.items()}
    s4 = hhg.Shell(0.55, 1.0, 0, 1, 4)
    s5 = hhg.Shell(0.55, 1.0, 0, 1, 5)
    yield levels, As, s4, s5
    s4.close()
    s5.close()


@pytest.mark.parametrize("q,j,L", [(1, 2, 4), (3, 2, 4), (2, 1, 4), (2, 3, 5)])
def test_degree_and_sampling(setup, q, j, L):
    levels, As, s4, s5 = setup
    s = s4 if L == 4 else s5
    s.fit(q, j)
    for l2 in range(3, L + 1):
        lv, A = levels[l2], As[l2]
        B = LS.surrogate_operator(lv, A, LS.fit(lv, A, q, j), q)
        op = mg.Operator(lv, B)
        u = synthetic.uniform(lv.n_total, synthetic.SEED_U)
        f = synthetic.uniform(lv.n_total, synthetic.SEED_F)
        ut, ft = torch.from_numpy(u).cuda(), torch.from_numpy(f).cuda()
        y = torch.empty_like(ut)
        s.apply(ut, y, L=l2, op=hhg.HHG_OP_LSQP)
        us = ut.clone()
        s.smooth(ft, us, 1, L=l2, op=hhg.HHG_OP_LSQP)
        u32 = u.astype(np.float32)
        y32 = torch.empty(lv.n_total, dtype=torch.float32, device="cuda")
        s.apply(torch.from_numpy(u32).cuda(), y32, L=l2, op=hhg.HHG_OP_LSQP, dtype=hhg.HHG_F32)
        torch.cuda.synchronize()
        assert rel(y.cpu().numpy(), op.apply(u), lv.free) <= 1e-12
        assert rel(us.cpu().numpy(), op.sweep(op.mask * u, f), lv.free) <= 1e-12
        assert rel(y32.cpu().numpy().astype(np.float64), op.apply(u32.astype(np.float64)), lv.free) <= TOL32


@pytest.mark.parametrize("q", [1, 3])
def test_ipoly_degree(setup, q):
    """IPOLY of degree 1 and 3 (hhg_fit_ipoly_degree): FP64 apply and one
    sweep against the oracle's IPOLY surrogate at N = 8 and 16 to 1e-12."""
    levels, As, s4, _ = setup
    s4.fit_ipoly(q)
    for l2 in (3, 4):
        lv, A = levels[l2], As[l2]
        op = mg.Operator(lv, LS.surrogate_operator(lv, A, LS.fit_ipoly(lv, A, q=q), q))
        u = synthetic.uniform(lv.n_total, synthetic.SEED_U)
        f = synthetic.uniform(lv.n_total, synthetic.SEED_F)
        ut, ft = torch.from_numpy(u).cuda(), torch.from_numpy(f).cuda()
        y = torch.empty_like(ut)
        s4.apply(ut, y, L=l2, op=hhg.HHG_OP_LSQP)
        us = ut.clone()
        s4.smooth(ft, us, 1, L=l2, op=hhg.HHG_OP_LSQP)
        torch.cuda.synchronize()
        assert rel(y.cpu().numpy(), op.apply(u), lv.free) <= 1e-12
        assert rel(us.cpu().numpy(), op.sweep(op.mask * u, f), lv.free) <= 1e-12
