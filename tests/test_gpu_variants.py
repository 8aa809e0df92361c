"""Method variants of the paper on the GPU against the FP64 oracle (60-macro
shell, N = 16): IPOLY (Sec. 3.1, quadratic interpolation at ten points per
macro cell) as operator and in V-cycles, and double discretisation (Sec. 4.1:
surrogate relaxation, exact residuals, stopping on the updates).  Bars as
for LSQP: 1e-12 relative for an operator application, 1e-10 for V-cycle
iterates (CG vs direct coarse solve)."""
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

L = 4


def rel(a, b, free):
    return np.linalg.norm(a[free] - b[free]) / np.linalg.norm(b[free])


@pytest.fixture(scope="module")
def shell():
    sh = M.make_shell()
    s = hhg.Shell(0.55, 1.0, 0, 1, L)
    yield sh, s
    s.close()


def test_ipoly_apply_matches_oracle(shell):
    sh, s = shell
    s.fit_ipoly()
    for l2 in (3, 4):
        lv = M.make_level(sh, 2 ** l2)
        A = F.assemble(lv)
        B = LS.surrogate_operator(lv, A, LS.fit_ipoly(lv, A), 2)
        u = synthetic.uniform(lv.n_total, synthetic.SEED_U)
        y = torch.empty(lv.n_total, dtype=torch.float64, device="cuda")
        s.apply(torch.from_numpy(u).cuda(), y, L=l2, op=hhg.HHG_OP_LSQP)
        torch.cuda.synchronize()
        ref = mg.Operator(lv, B).apply(u)
        assert rel(y.cpu().numpy(), ref, lv.free) <= 1e-12


@pytest.mark.parametrize("kind", ["ipoly", "dd-lsqp", "dd-ipoly"])
def test_variant_cycles_match_oracle(shell, kind):
    sh, s = shell
    if kind.endswith("ipoly"):
        s.fit_ipoly()
    else:
        s.fit(2, 2)
    op = hhg.HHG_OP_DD if kind.startswith("dd-") else hhg.HHG_OP_LSQP
    H = mg.build_hierarchy(sh, 2 ** L, kind)
    lv = H.levels[-1]
    f = synthetic.uniform(lv.n_total, synthetic.SEED_F)
    u = np.zeros(lv.n_total)
    ft = torch.from_numpy(f).cuda()
    ut = torch.zeros_like(ft)
    for _ in range(2):
        u = H.vcycle(len(H.ops) - 1, u, f)
    s.vcycle(ft, ut, max_cycles=2, rtol=0.0, op=op, raise_on_noconv=False)
    torch.cuda.synchronize()
    assert rel(ut.cpu().numpy(), u, lv.free) <= 1e-10


def test_dd_stops_on_updates_like_the_oracle(shell):
    sh, s = shell
    s.fit(2, 2)
    H = mg.build_hierarchy(sh, 2 ** L, "dd-lsqp")
    lv = H.levels[-1]
    f = synthetic.uniform(lv.n_total, synthetic.SEED_F)
    u_ref, hist = H.solve_updates(f, rtol=1e-8, max_cycles=40)
    ft = torch.from_numpy(f).cuda()
    ut = torch.zeros_like(ft)
    relres, cycles, _ = s.vcycle(ft, ut, rtol=1e-8, op=hhg.HHG_OP_DD, max_cycles=40)
    torch.cuda.synchronize()
    assert relres[0] <= 1e-8
    assert abs(cycles - len(hist)) <= 1
    assert rel(ut.cpu().numpy(), u_ref, lv.free) <= 1e-7


def test_dd_mixed_precision_is_defect_correction(shell):
    """Double discretisation inside mixed-precision refinement: the FP64
    outer loop forms the exact residual f - L u every cycle and the FP32
    cycle relaxes with the surrogate, so the refinement's fixed point is the
    solution of the exact operator (defect correction), not the fixed point
    of the FP64 double-discretisation cycle.  It reaches the update tolerance
    and the exact (IFEM) FP64 solution to 1e-6; the oracle's defect
    correction with its FP64 DD cycle shows the same fixed point (7e-13 from
    the exact solution, 0.7 % from the DD iterate on this shell)."""
    sh, s = shell
    s.fit(2, 2)
    n, _ = s.num_nodes()
    f = torch.from_numpy(synthetic.uniform(n, synthetic.SEED_F)).cuda()
    ue, u32 = torch.zeros_like(f), torch.zeros_like(f)
    rele, _, _ = s.vcycle(f, ue, rtol=1e-11, op=hhg.HHG_OP_IFEM, dtype=hhg.HHG_F64, max_cycles=60)
    rel32, _, _ = s.vcycle(f, u32, rtol=1e-9, op=hhg.HHG_OP_DD, dtype=hhg.HHG_F32, max_cycles=60)
    torch.cuda.synchronize()
    assert rele[0] <= 1e-11 and rel32[0] <= 1e-9
    free = M.make_level(sh, 2 ** L).free
    assert rel(u32.cpu().numpy(), ue.cpu().numpy(), free) <= 1e-6
