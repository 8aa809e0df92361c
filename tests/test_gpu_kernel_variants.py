"""The kernels of the surrogate smoother, apply and residual give the same
bits (Sec. 3.4).

FP64: the per-node kernel (the default) evaluates each weight by integer
Horner from the plane table; the run kernels take a run of up to 8 points of
one line per thread and reach every weight by exact integer forward
differences along the run (Eq. 5.4 in exact arithmetic); the cell-resident
sweep runs the four colour steps of a cell on its interior held in the
shared memory of a thread-block cluster (2 CTAs at N = 64).  All form the
same integers, convert them the same way and apply them in the same order,
so apply, residual, smoother sweeps and whole V-cycles must agree bit for
bit; the residual norms are sums in another order and agree to 1e-14.
Shells of 60 cells at N = 8, 16, 32 and of 480 cells at N = 64 (runs of
every length, lines with only boundary-adjacent points, all three degrees
q).

FP32: the cell-resident sweep (tuner configuration 7; clusters of 1 CTA up
to N = 64 and of 8 CTAs at N = 128, where neighbours on the adjacent slab's
planes come from another CTA's shared memory) against the per-colour
thread-per-node kernel (configuration -1), bit for bit.

Parity of the default kernels with the oracle is covered by the other GPU
tests."""
import numpy as np
import pytest

import synthetic

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1608_06473_gb300 as hhg  # noqa: E402

CASES = [(0, 1, 3), (0, 1, 4), (0, 1, 5), (1, 2, 6)]


def _vectors(n):
    u = torch.from_numpy(synthetic.uniform(n, synthetic.SEED_U)).cuda()
    f = torch.from_numpy(synthetic.uniform(n, synthetic.SEED_F)).cuda()
    return u, f


def _run_all(s, variant, u, f):
    hhg.hhg_set_fp64_kernel(s.handle, variant)
    y, r, us = torch.empty_like(u), torch.empty_like(u), u.clone()
    s.apply(u, y)
    norm = s.residual(u, f, r)[0]
    s.smooth(f, us, 2)
    uv = torch.zeros_like(u)
    s.vcycle(f, uv, max_cycles=2, rtol=0.0, raise_on_noconv=False)
    torch.cuda.synchronize()
    return y, r, norm, us, uv


@pytest.mark.parametrize("tang,layers,L", CASES)
@pytest.mark.parametrize("q", [1, 2, 3])
def test_runs_equal_nodes_bitwise(tang, layers, L, q):
    with hhg.Shell(0.55, 1.0, tang, layers, L) as s:
        s.fit(q, 2)
        n, _ = s.num_nodes()
        u, f = _vectors(n)
        a = _run_all(s, hhg.FP64_NODES, u, f)
        for variant in (hhg.FP64_RUNS, hhg.FP64_RESIDENT):
            b = _run_all(s, variant, u, f)
            for name, x, z in zip(("apply", "residual", "smoother", "V-cycles"), a[:2] + a[3:], b[:2] + b[3:]):
                assert torch.equal(x, z), f"{name}: variant {variant} and the nodes kernel differ (q={q}, N={2 ** L})"
            assert abs(a[2] - b[2]) <= 1e-14 * abs(a[2])


@pytest.mark.parametrize("L", [4, 5, 6, 7])
@pytest.mark.parametrize("q", [1, 2, 3])
def test_fp32_resident_equals_node_kernel_bitwise(L, q):
    with hhg.Shell(0.55, 1.0, 0, 1, L) as s:
        s.fit(q, 2)
        n, _ = s.num_nodes()
        u, f = _vectors(n)
        u, f = u.float(), f.float()
        s.smooth(f, u.clone(), 1, op=hhg.HHG_OP_LSQP, dtype=hhg.HHG_F32)   # FP32 buffers and the tuner's run
        out = {}
        for cfg in (-1, 7):
            hhg.hhg_set_tuning(s.handle, L, cfg)
            us = u.clone()
            s.smooth(f, us, 2, op=hhg.HHG_OP_LSQP, dtype=hhg.HHG_F32)
            torch.cuda.synchronize()
            out[cfg] = us
        assert torch.equal(out[-1], out[7]), f"FP32 resident sweep differs from the node kernel (q={q}, N={2 ** L})"


def test_unknown_variant_rejected():
    with hhg.Shell(0.55, 1.0, 0, 1, 3) as s:
        with pytest.raises(hhg.HHGError):
            hhg.hhg_set_fp64_kernel(s.handle, 7)


def test_run_lists_cover_every_interior_point_once():
    """The run lists are read only on the device; this checks them through
    their effect: a residual with f = 0 on a vector that is 1 at every free
    node gives exactly the apply's negation at every interior node."""
    with hhg.Shell(0.55, 1.0, 0, 1, 5) as s:
        s.fit(2, 2)
        n, _ = s.num_nodes()
        u = torch.ones(n, dtype=torch.float64, device="cuda")
        f = torch.zeros_like(u)
        y, r = torch.full_like(u, np.nan), torch.full_like(u, np.nan)
        s.apply(u, y)
        s.residual(u, f, r)
        torch.cuda.synchronize()
        assert not torch.isnan(y).any() and not torch.isnan(r).any()
        assert torch.equal(r, -y)
