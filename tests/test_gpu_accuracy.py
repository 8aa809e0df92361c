"""The accuracy study of Sec. 4 on the GPU against the FP64 oracle (60-cell
shell, N = 16): the vertex-quadrature load vector (hhg_load_vector) on the
blended and on the unprojected mesh to 1e-13 relative, CONS DD cycles
(hhg_fit_cons + HHG_OP_DD) to 1e-10, and the discrete L2 error after 10
V(3,3) cycles for FEM, LSQP, LSQP DD and CONS to 1e-9 relative."""
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
R1, R2 = 0.55, 1.0


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def shells():
    s = hhg.Shell(R1, R2, 0, 1, L)
    c = hhg.Shell(R1, R2, 0, 1, L, unprojected=True)
    yield s, c
    s.close()
    c.close()


@pytest.mark.parametrize("mapped", [True, False])
def test_load_vector_matches_oracle(shells, mapped):
    s = shells[0] if mapped else shells[1]
    sh = M.make_shell(R1, R2)
    for l2 in (2, 3, 4):
        lv = M.make_level(sh, 2 ** l2, mapped=mapped)
        _, fb = synthetic.manufactured(lv.coords, R1, R2)
        ref = F.load_vector(lv, fb)
        b = torch.full((lv.n_total,), np.nan, dtype=torch.float64, device="cuda")
        s.load_vector(torch.from_numpy(fb).cuda(), b, L=l2)
        torch.cuda.synchronize()
        got = b.cpu().numpy()
        assert rel(got, ref) <= 1e-13
        assert np.all(got[ref == 0] == 0)
    # host arrays in and out
    bh = np.empty(lv.n_total)
    s.load_vector(fb, bh, L=L)
    assert rel(bh, ref) <= 1e-13


def test_cons_dd_cycles_match_oracle(shells):
    s, _ = shells
    s.fit_cons(2, 2)
    sh = M.make_shell(R1, R2)
    H = mg.build_hierarchy(sh, 2 ** L, "dd-cons")
    lv = H.levels[-1]
    f = synthetic.uniform(lv.n_total, synthetic.SEED_F)
    u = np.zeros(lv.n_total)
    for _ in range(2):
        u = H.vcycle(len(H.ops) - 1, u, f)
    ft = torch.from_numpy(f).cuda()
    ut = torch.zeros_like(ft)
    s.vcycle(ft, ut, max_cycles=2, rtol=0.0, op=hhg.HHG_OP_DD, raise_on_noconv=False)
    torch.cuda.synchronize()
    assert rel(ut.cpu().numpy()[lv.free], u[lv.free]) <= 1e-10


@pytest.mark.parametrize("variant", ["fem", "lsqp", "dd-lsqp", "cons"])
def test_discretisation_error_matches_oracle(shells, variant):
    s = shells[1] if variant == "cons" else shells[0]
    sh = M.make_shell(R1, R2)
    kind = {"fem": "ifem", "lsqp": "lsqp", "dd-lsqp": "dd-lsqp", "cons": "ifem"}[variant]
    H = mg.build_hierarchy(sh, 2 ** L, kind, mapped=variant != "cons")
    lv = H.levels[-1]
    ub, fb = synthetic.manufactured(lv.coords, R1, R2)
    b = F.load_vector(lv, fb)
    u = np.zeros(lv.n_total)
    for _ in range(10):
        u = H.vcycle(len(H.ops) - 1, u, b)
    e_ref = F.discretisation_error(lv, ub, u)

    if variant in ("lsqp", "dd-lsqp"):
        s.fit(2, 2)
    op = {"fem": hhg.HHG_OP_IFEM, "lsqp": hhg.HHG_OP_LSQP, "dd-lsqp": hhg.HHG_OP_DD,
          "cons": hhg.HHG_OP_IFEM}[variant]
    X = s.node_coords()
    assert np.allclose(X, lv.coords, rtol=0, atol=1e-14)
    ug, fg = synthetic.manufactured(torch.from_numpy(X).cuda(), R1, R2, xp=torch)
    bt = torch.empty_like(fg)
    s.load_vector(fg, bt)
    ut = torch.zeros_like(bt)
    s.vcycle(bt, ut, max_cycles=10, rtol=0.0, op=op, raise_on_noconv=False)
    torch.cuda.synchronize()
    e_gpu = (1.0 / 2 ** L) ** 1.5 * float(torch.linalg.vector_norm(ug - ut))
    assert abs(e_gpu / e_ref - 1) <= 1e-9
