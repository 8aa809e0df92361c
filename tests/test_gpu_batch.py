"""Batched right-hand sides: with all vectors in device memory, nrhs vectors
go through every kernel together (the surrogate weights of a node are
evaluated once for the whole group).  Each result must equal the
one-vector-at-a-time result: apply, residual and smoother to 1e-13 relative
in FP64 (the same arithmetic per vector) and to the FP32 bound in FP32; a
fixed number of V-cycles to 1e-10 in FP64 and 1e-6 in mixed precision (the
batched coarse conjugate-gradient solve iterates until every vector has
converged, so converged vectors take extra iterations; in mixed precision
those last-digit changes of the FP64 coarse correction flip FP32 roundings
of the inner cycle); a batched solve reaches 1e-8 for every vector and
agrees with the oracle's V-cycle on one of them.  The cell kernels form a
node's weights once for all right-hand sides of the call; nrhs = 32 (the
batched configuration's count) is checked per vector against single calls:
bitwise in FP64 for the surrogate apply and smoother (the same integer
weights and the same FMA order), 1e-13 for IFEM and the residual norms, the
FP32 bound in FP32."""
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

NRHS = 5
OPS = {"ifem": hhg.HHG_OP_IFEM, "lsqp": hhg.HHG_OP_LSQP}
TOL = {hhg.HHG_F64: 1e-13, hhg.HHG_F32: 2e-5}


@pytest.fixture(scope="module")
def c1():
    sh = M.make_shell()
    s = hhg.Shell(0.55, 1.0, 0, 1, 4)
    s.fit(2, 2)
    n_total, _ = s.num_nodes()
    lv = M.make_level(sh, 16)
    yield s, n_total, lv
    s.close()


def rel(a, b, free):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return np.linalg.norm(a[:, free] - b[:, free]) / np.linalg.norm(b[:, free])


def vectors(n, dt):
    U = synthetic.batch(n, NRHS)
    Fv = synthetic.batch(n, NRHS, "gaussian")
    return torch.from_numpy(U.astype(dt)).cuda(), torch.from_numpy(Fv.astype(dt)).cuda()


@pytest.mark.parametrize("dtype", [hhg.HHG_F64, hhg.HHG_F32])
@pytest.mark.parametrize("opname", ["lsqp", "ifem"])
def test_batched_operators_match_single(c1, opname, dtype):
    s, n, lv = c1
    op = OPS[opname]
    dt = np.float64 if dtype == hhg.HHG_F64 else np.float32
    U, Fv = vectors(n, dt)
    Y, R = torch.empty_like(U), torch.empty_like(U)
    s.apply(U, Y, op=op, dtype=dtype, nrhs=NRHS)
    norms = s.residual(U, Fv, R, op=op, dtype=dtype, nrhs=NRHS)
    Us = U.clone()
    s.smooth(Fv, Us, 2, op=op, dtype=dtype, nrhs=NRHS)
    torch.cuda.synchronize()
    y1, r1, s1, n1 = [], [], [], []
    for b in range(NRHS):
        y, r, u = torch.empty_like(U[b]), torch.empty_like(U[b]), U[b].clone()
        s.apply(U[b], y, op=op, dtype=dtype)
        n1.append(s.residual(U[b], Fv[b], r, op=op, dtype=dtype)[0])
        s.smooth(Fv[b], u, 2, op=op, dtype=dtype)
        y1.append(y)
        r1.append(r)
        s1.append(u)
    torch.cuda.synchronize()
    tol = TOL[dtype]
    st = lambda xs: torch.stack(xs).cpu().numpy()
    assert rel(Y.cpu().numpy(), st(y1), lv.free) <= tol
    assert rel(R.cpu().numpy(), st(r1), lv.free) <= tol
    assert rel(Us.cpu().numpy(), st(s1), lv.free) <= tol
    assert np.allclose(norms, n1, rtol=max(tol, 1e-12))


@pytest.mark.parametrize("dtype", [hhg.HHG_F64, hhg.HHG_F32])
@pytest.mark.parametrize("opname", ["lsqp", "ifem"])
def test_batched_32_match_single(c1, opname, dtype):
    s, n, lv = c1
    op = OPS[opname]
    nb = 32
    dt = np.float64 if dtype == hhg.HHG_F64 else np.float32
    U = torch.from_numpy(synthetic.batch(n, nb).astype(dt)).cuda()
    Fv = torch.from_numpy(synthetic.batch(n, nb, "gaussian").astype(dt)).cuda()
    Y, R, Us = torch.empty_like(U), torch.empty_like(U), U.clone()
    s.apply(U, Y, op=op, dtype=dtype, nrhs=nb)
    norms = s.residual(U, Fv, R, op=op, dtype=dtype, nrhs=nb)
    s.smooth(Fv, Us, 1, op=op, dtype=dtype, nrhs=nb)
    torch.cuda.synchronize()
    exact = dtype == hhg.HHG_F64 and opname == "lsqp"
    for b in (0, 7, 31):
        y, r, u = torch.empty_like(U[b]), torch.empty_like(U[b]), U[b].clone()
        s.apply(U[b], y, op=op, dtype=dtype)
        nr = s.residual(U[b], Fv[b], r, op=op, dtype=dtype)[0]
        s.smooth(Fv[b], u, 1, op=op, dtype=dtype)
        torch.cuda.synchronize()
        for got, ref in ((Y[b], y), (R[b], r), (Us[b], u)):
            g, e = got.cpu().numpy()[None], ref.cpu().numpy()[None]
            if exact:
                assert np.array_equal(g[:, lv.free], e[:, lv.free])
            else:
                assert rel(g, e, lv.free) <= TOL[dtype]
        assert abs(norms[b] - nr) <= max(TOL[dtype], 1e-13) * nr


@pytest.mark.parametrize("dtype", [hhg.HHG_F64, hhg.HHG_F32])
def test_batched_cycles_match_single(c1, dtype):
    s, n, lv = c1
    _, Fv = vectors(n, np.float64)
    U = torch.zeros_like(Fv)
    s.vcycle(Fv, U, max_cycles=2, rtol=0.0, dtype=dtype, nrhs=NRHS, raise_on_noconv=False)
    ref = []
    for b in range(NRHS):
        u = torch.zeros_like(Fv[b])
        s.vcycle(Fv[b], u, max_cycles=2, rtol=0.0, dtype=dtype, raise_on_noconv=False)
        ref.append(u)
    torch.cuda.synchronize()
    tol = 1e-10 if dtype == hhg.HHG_F64 else 1e-6
    assert rel(U.cpu().numpy(), torch.stack(ref).cpu().numpy(), lv.free) <= tol


def test_batched_solve_converges_and_matches_oracle(c1):
    s, n, lv = c1
    _, Fv = vectors(n, np.float64)
    U = torch.zeros_like(Fv)
    relres, cycles, _ = s.vcycle(Fv, U, rtol=1e-8, nrhs=NRHS)
    assert np.all(relres <= 1e-8)
    # the oracle's V(3,3) on right-hand side 2, same number of cycles
    sh = M.make_shell()
    levels, ops = [], []
    for l2 in range(2, 5):
        lvl = M.make_level(sh, 2 ** l2)
        A = F.assemble(lvl)
        if l2 >= 3:
            A = LS.surrogate_operator(lvl, A, LS.fit(lvl, A, 2, 2), 2)
        levels.append(lvl)
        ops.append(mg.Operator(lvl, A))
    H = mg.Hierarchy(levels, ops)
    f2 = Fv[2].cpu().numpy()
    u = np.zeros(n)
    for _ in range(cycles):
        u = H.vcycle(len(ops) - 1, u, f2)
    got = U[2].cpu().numpy()
    fr = lv.free
    assert np.linalg.norm(got[fr] - u[fr]) / np.linalg.norm(u[fr]) <= 1e-9


@pytest.mark.parametrize("dtype", [hhg.HHG_F64, hhg.HHG_F32])
def test_graph_cycles_match_launch_by_launch(c1, dtype):
    """Cycles replayed from a CUDA graph (fixed-count coarse iterations)
    against the same number of cycles launched one by one: the iterates agree
    to the coarse solve's tolerance (1e-10 FP64; 1e-6 mixed, whose FP32
    roundings react to last-digit changes of the coarse correction), and a
    graph-replayed solve reaches 1e-8."""
    s, n, lv = c1
    _, Fv = vectors(n, np.float64)
    out = {}
    for graphs in (False, True):
        hhg.hhg_set_graphs(s.handle, graphs)
        U = torch.zeros_like(Fv)
        s.vcycle(Fv, U, max_cycles=4, rtol=0.0, dtype=dtype, nrhs=NRHS, raise_on_noconv=False)
        torch.cuda.synchronize()
        out[graphs] = U.cpu().numpy()
    tol = 1e-10 if dtype == hhg.HHG_F64 else 1e-6
    assert rel(out[True], out[False], lv.free) <= tol
    U = torch.zeros_like(Fv)
    relres, _, _ = s.vcycle(Fv, U, rtol=1e-8, dtype=dtype, nrhs=NRHS)
    assert np.all(relres <= 1e-8)
