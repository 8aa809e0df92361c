"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on the
same seeded inputs.  Bar (FP64): ||x_gpu - x_oracle||_2 <= 1e-12 ||x_oracle||_2
over the unknowns, for operator application, residual and one smoother sweep;
the V-cycle differs only through the coarse solve (GPU conjugate gradients to
1e-13 vs the oracle's sparse direct solve), bounded by 1e-10."""
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

TOL = 1e-12


def rel_err(got, ref, free):
    return np.linalg.norm(got[free] - ref[free]) / np.linalg.norm(ref[free])


class OracleShell:
    """Oracle operators on all levels of one shell, built once per module."""

    def __init__(self, tang, layers, L, q=2, j=2):
        self.sh = M.make_shell(tang=tang, layers=layers)
        self.levels, self.exact, self.surr = {}, {}, {}
        for l2 in range(2, L + 1):
            lv = M.make_level(self.sh, 2 ** l2)
            A = F.assemble(lv)
            self.levels[l2] = lv
            self.exact[l2] = A
            self.surr[l2] = LS.surrogate_operator(lv, A, LS.fit(lv, A, q, j), q) if l2 >= 3 else A

    def op(self, L, opname):
        return mg.Operator(self.levels[L], self.surr[L] if opname == "lsqp" else self.exact[L])

    def hierarchy(self, opname):
        Ls = sorted(self.levels)
        return mg.Hierarchy([self.levels[l] for l in Ls], [self.op(l, opname) for l in Ls])


@pytest.fixture(scope="module")
def c1():
    ora = OracleShell(0, 1, 4)
    s = hhg.Shell(0.55, 1.0, 0, 1, 4)
    s.fit(2, 2)
    torch.cuda.synchronize()
    yield ora, s
    s.close()


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


OPS = {"ifem": hhg.HHG_OP_IFEM, "lsqp": hhg.HHG_OP_LSQP}


def test_node_counts_and_coords(c1):
    ora, s = c1
    for L in (2, 3, 4):
        lv = ora.levels[L]
        assert s.num_nodes(L) == (lv.n_total, int((~lv.dirichlet).sum()))
        assert np.max(np.abs(s.node_coords(L) - lv.coords)) <= 1e-15


@pytest.mark.parametrize("opname", ["ifem", "lsqp"])
@pytest.mark.parametrize("L", [2, 3, 4])
def test_apply(c1, opname, L):
    ora, s = c1
    lv = ora.levels[L]
    u = synthetic.uniform(lv.n_total, synthetic.SEED_U)
    y = torch.zeros(lv.n_total, dtype=torch.float64, device="cuda")
    s.apply(dev(u), y, L=L, op=OPS[opname])
    ref = ora.op(L, opname).apply(u)
    got = host(y)
    assert rel_err(got, ref, lv.free) <= TOL
    assert np.all(got[lv.dirichlet] == 0)


@pytest.mark.parametrize("opname", ["ifem", "lsqp"])
def test_residual_and_norm(c1, opname):
    ora, s = c1
    L = 4
    lv = ora.levels[L]
    u = synthetic.uniform(lv.n_total, synthetic.SEED_U)
    f = synthetic.uniform(lv.n_total, synthetic.SEED_F)
    r = torch.zeros(lv.n_total, dtype=torch.float64, device="cuda")
    norms = s.residual(dev(u), dev(f), r, L=L, op=OPS[opname])
    ref = ora.op(L, opname).residual(u, f)
    got = host(r)
    assert rel_err(got, ref, lv.free) <= TOL
    assert abs(norms[0] - np.linalg.norm(ref)) <= TOL * np.linalg.norm(ref)
    assert abs(norms[0] - np.linalg.norm(got)) <= 1e-14 * np.linalg.norm(got)


@pytest.mark.parametrize("opname", ["ifem", "lsqp"])
@pytest.mark.parametrize("sweeps", [1, 2])
def test_smoother(c1, opname, sweeps):
    ora, s = c1
    L = 4
    lv = ora.levels[L]
    u0 = synthetic.uniform(lv.n_total, synthetic.SEED_U)
    f = synthetic.uniform(lv.n_total, synthetic.SEED_F)
    ut = dev(u0)
    s.smooth(dev(f), ut, sweeps=sweeps, L=L, op=OPS[opname])
    op = ora.op(L, opname)
    ref = u0 * op.mask
    for _ in range(sweeps):
        ref = op.sweep(ref, f)
    got = host(ut)
    assert rel_err(got, ref, lv.free) <= TOL
    assert np.all(got[lv.dirichlet] == 0)


@pytest.mark.parametrize("opname", ["ifem", "lsqp"])
def test_vcycle_history(c1, opname):
    ora, s = c1
    H = ora.hierarchy(opname)
    lv = ora.levels[4]
    f = synthetic.uniform(lv.n_total, synthetic.SEED_F)
    u_ref = np.zeros(lv.n_total)
    op = H.ops[-1]
    r0 = np.linalg.norm(op.residual(u_ref, f))
    ut = torch.zeros(lv.n_total, dtype=torch.float64, device="cuda")
    ft = dev(f)
    for cyc in range(3):
        u_ref = H.vcycle(len(H.ops) - 1, u_ref, f)
        s.vcycle(ft, ut, max_cycles=1, rtol=0.0, op=OPS[opname], raise_on_noconv=False)
        got = host(ut)
        assert rel_err(got, u_ref, lv.free) <= 1e-10
        r = torch.zeros_like(ut)
        nrm = s.residual(ut, ft, r, op=OPS[opname])[0]
        ref_n = np.linalg.norm(op.residual(u_ref, f))
        assert abs(nrm - ref_n) / r0 <= 1e-10


@pytest.mark.parametrize("opname", ["ifem", "lsqp"])
def test_solve_to_1e8(c1, opname):
    ora, s = c1
    H = ora.hierarchy(opname)
    lv = ora.levels[4]
    f = synthetic.uniform(lv.n_total, synthetic.SEED_F)
    u_ref, hist = H.solve(f, rtol=1e-8)
    ut = torch.zeros(lv.n_total, dtype=torch.float64, device="cuda")
    rel, cycles, st = s.vcycle(dev(f), ut, rtol=1e-8, op=OPS[opname])
    assert rel[0] <= 1e-8
    assert cycles == len(hist) - 1
    assert abs(rel[0] - hist[-1]) <= 1e-6 * hist[-1]
    assert rel_err(host(ut), u_ref, lv.free) <= 1e-9


def test_host_pointer_arguments_match_device(c1):
    ora, s = c1
    lv = ora.levels[4]
    f = synthetic.uniform(lv.n_total, synthetic.SEED_F)
    u_host = np.zeros(lv.n_total)
    s.vcycle(f, u_host, max_cycles=2, rtol=0.0, raise_on_noconv=False)
    ut = torch.zeros(lv.n_total, dtype=torch.float64, device="cuda")
    s.vcycle(dev(f), ut, max_cycles=2, rtol=0.0, raise_on_noconv=False)
    assert np.array_equal(u_host, host(ut))
    y_host = np.zeros(lv.n_total)
    s.apply(f, y_host)
    yt = torch.zeros_like(ut)
    s.apply(dev(f), yt)
    assert np.array_equal(y_host, host(yt))


def test_errors():
    with pytest.raises(hhg.HHGError) as e:
        hhg.Shell(0.55, 1.0, 0, 1, 1)
    assert e.value.status == hhg.Status.EINVAL
    with pytest.raises(hhg.HHGError) as e:
        hhg.Shell(0.55, 1.0, 0, 1, 4, hbm_budget_bytes=1 << 16)
    assert e.value.status == hhg.Status.ENOMEM
    s = hhg.Shell(0.55, 1.0, 0, 1, 3)
    try:
        n, _ = s.num_nodes()
        y = torch.zeros(n, dtype=torch.float64, device="cuda")
        u = torch.ones(n, dtype=torch.float64, device="cuda")
        with pytest.raises(hhg.HHGError) as e:
            s.apply(u, y, op=hhg.HHG_OP_LSQP)
        assert e.value.status == hhg.Status.ENOTFIT
        with pytest.raises(hhg.HHGError) as e:
            s.apply(u, y, L=5)
        assert e.value.status == hhg.Status.EINVAL
        s.apply(u, y, op=hhg.HHG_OP_IFEM)
        # constants lie in the kernel of the operator away from the boundary
        got = host(y)
        assert np.abs(got).max() < 1e3
    finally:
        s.close()
