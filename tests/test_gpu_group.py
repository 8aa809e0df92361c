"""Several shells of differing radius ratio in one hierarchy (hhg_setup_shells):
the shells become disjoint components of one macro mesh, so each kernel
launch spans all of them.  Every shell's part of a group result must equal
the same operation on that shell alone -- apply and one smoother sweep to
1e-13 relative (the same arithmetic per node), fixed V-cycles to 1e-10 (the
coarse conjugate-gradient solve iterates on the whole group) -- and one
shell's part agrees with the FP64 oracle; a group sweep launches as many
kernels as a single-shell sweep."""
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

RADII = [(0.35, 1.0), (0.55, 1.0), (0.7, 1.0)]
L = 4


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def shells():
    g = hhg.Shell.group(RADII, fine_log2_intervals=L)
    g.fit(2, 2)
    singles = []
    for ri, ro in RADII:
        s = hhg.Shell(ri, ro, 0, 1, L)
        s.fit(2, 2)
        singles.append(s)
    yield g, singles
    g.close()
    for s in singles:
        s.close()


def split(g, vec, k, Lv=L):
    return vec[g.part_index(k, Lv)]


def test_layout_partitions_the_group(shells):
    g, singles = shells
    n_tot = sum(s.num_nodes()[0] for s in singles)
    assert g.num_nodes()[0] == n_tot
    idx = np.concatenate([g.part_index(k) for k in range(len(RADII))])
    assert np.array_equal(np.sort(idx), np.arange(n_tot))


def test_group_apply_and_sweep_equal_single_shells(shells):
    g, singles = shells
    n = g.num_nodes()[0]
    u = synthetic.uniform(n, synthetic.SEED_U)
    f = synthetic.uniform(n, synthetic.SEED_F)
    ut, ft = torch.from_numpy(u).cuda(), torch.from_numpy(f).cuda()
    y = torch.empty_like(ut)
    g.apply(ut, y)
    us = ut.clone()
    l0 = hhg.hhg_launch_count()
    g.smooth(ft, us, 1)
    torch.cuda.synchronize()
    launches_group = hhg.hhg_launch_count() - l0
    yh, sh = y.cpu().numpy(), us.cpu().numpy()
    for k, s in enumerate(singles):
        uk = torch.from_numpy(split(g, u, k)).cuda()
        fk = torch.from_numpy(split(g, f, k)).cuda()
        yk = torch.empty_like(uk)
        s.apply(uk, yk)
        l0 = hhg.hhg_launch_count()
        s.smooth(fk, uk, 1)
        torch.cuda.synchronize()
        assert hhg.hhg_launch_count() - l0 == launches_group
        assert rel(split(g, yh, k), yk.cpu().numpy()) <= 1e-13
        assert rel(split(g, sh, k), uk.cpu().numpy()) <= 1e-13


def test_group_cycles_equal_single_shells_and_oracle(shells):
    g, singles = shells
    n = g.num_nodes()[0]
    f = synthetic.uniform(n, synthetic.SEED_F)
    ft = torch.from_numpy(f).cuda()
    ut = torch.zeros_like(ft)
    g.vcycle(ft, ut, max_cycles=2, rtol=0.0, raise_on_noconv=False)
    torch.cuda.synchronize()
    uh = ut.cpu().numpy()
    for k, s in enumerate(singles):
        fk = torch.from_numpy(split(g, f, k)).cuda()
        uk = torch.zeros_like(fk)
        s.vcycle(fk, uk, max_cycles=2, rtol=0.0, raise_on_noconv=False)
        torch.cuda.synchronize()
        assert rel(split(g, uh, k), uk.cpu().numpy()) <= 1e-10
    # shell 0 (r in [0.35, 1]) against the oracle's V(3,3)
    sh = M.make_shell(r1=RADII[0][0], r2=RADII[0][1])
    levels, ops = [], []
    for l2 in range(2, L + 1):
        lv = M.make_level(sh, 2 ** l2)
        A = F.assemble(lv)
        if l2 >= 3:
            A = LS.surrogate_operator(lv, A, LS.fit(lv, A, 2, 2), 2)
        levels.append(lv)
        ops.append(mg.Operator(lv, A))
    H = mg.Hierarchy(levels, ops)
    f0 = split(g, f, 0)
    u = np.zeros_like(f0)
    for _ in range(2):
        u = H.vcycle(len(ops) - 1, u, f0)
    fr = levels[-1].free
    assert rel(split(g, uh, 0)[fr], u[fr]) <= 1e-10
