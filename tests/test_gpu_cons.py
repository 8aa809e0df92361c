"""The CONS operator (Sec. 4.1): the P1 stiffness on the unprojected
polyhedral domain Omega_H (Phi = Id), built as an unprojected shell.  Against
the FP64 oracle's assembly on the unmapped levels: node positions exactly,
apply to 1e-12, and V-cycles to 1e-10.  On straight macro cells every
interior stencil is constant per cell, so the surrogate fitted there
reproduces the exact operator (to rounding)."""
import numpy as np
import pytest

import synthetic
from oracle import fem as F
from oracle import mesh as M
from oracle import mg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1608_06473_gb300 as hhg  # noqa: E402

L = 4


def rel(a, b, free):
    return np.linalg.norm(a[free] - b[free]) / np.linalg.norm(b[free])


@pytest.fixture(scope="module")
def cons():
    sh = M.make_shell()
    s = hhg.Shell(0.55, 1.0, 0, 1, L, unprojected=True)
    s.fit(2, 2)
    levels = [M.make_level(sh, 2 ** l2, mapped=False) for l2 in range(2, L + 1)]
    ops = [mg.Operator(lv, F.assemble(lv)) for lv in levels]
    yield s, levels, ops
    s.close()


def test_nodes_stay_on_the_macro_mesh(cons):
    s, levels, _ = cons
    for l2, lv in zip(range(2, L + 1), levels):
        assert np.allclose(s.node_coords(l2), lv.coords, rtol=0, atol=1e-15)


@pytest.mark.parametrize("opname", ["ifem", "lsqp"])
def test_cons_apply(cons, opname):
    s, levels, ops = cons
    op = hhg.HHG_OP_IFEM if opname == "ifem" else hhg.HHG_OP_LSQP
    tol = 1e-12 if opname == "ifem" else 1e-11
    for l2, lv, o in zip(range(2, L + 1), levels, ops):
        u = synthetic.uniform(lv.n_total, synthetic.SEED_U)
        y = torch.empty(lv.n_total, dtype=torch.float64, device="cuda")
        s.apply(torch.from_numpy(u).cuda(), y, L=l2, op=op)
        torch.cuda.synchronize()
        assert rel(y.cpu().numpy(), o.apply(u), lv.free) <= tol


def test_cons_cycles(cons):
    s, levels, ops = cons
    H = mg.Hierarchy(levels, ops)
    lv = levels[-1]
    f = synthetic.uniform(lv.n_total, synthetic.SEED_F)
    u = np.zeros(lv.n_total)
    for _ in range(2):
        u = H.vcycle(len(ops) - 1, u, f)
    ft = torch.from_numpy(f).cuda()
    ut = torch.zeros_like(ft)
    s.vcycle(ft, ut, max_cycles=2, rtol=0.0, op=hhg.HHG_OP_IFEM, raise_on_noconv=False)
    torch.cuda.synchronize()
    assert rel(ut.cpu().numpy(), u, lv.free) <= 1e-10
