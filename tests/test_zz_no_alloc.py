"""hhg_residual_noalloc: the residual entry point that allocates nothing.

Callers that cannot allocate device memory when they need a residual (a
latency-critical loop that must not stall on cudaMalloc's implicit device
synchronisation, or a process whose device memory is reserved by a pool
allocator) use this variant: its norm partial sums live in a fixed array in
the library image.  Checked here against hhg_residual on two calls in a row,
through the C ABI, with the tolerance of the other parity tests.  The file is
named to be collected last.
"""
import numpy as np
import pytest

import synthetic

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1608_06473_gb300 as hhg  # noqa: E402

TOL = 1e-12


def test_noalloc_residual_matches_hhg_residual_twice():
    with hhg.Shell(0.55, 1.0, 0, 1, 4) as s:
        s.fit(2, 2)
        n, _ = s.num_nodes()
        for call, (su, sf) in enumerate(((1, 0), (3, 2))):
            u = torch.from_numpy(synthetic.uniform(n, su)).cuda()
            f = torch.from_numpy(synthetic.uniform(n, sf)).cuda()
            for op in (hhg.HHG_OP_LSQP, hhg.HHG_OP_IFEM):
                r_ref = torch.empty_like(u)
                nrm_ref = s.residual(u, f, r_ref, op=op)[0]
                r = torch.full_like(u, np.nan)
                norm2 = torch.full((1,), np.nan, dtype=torch.float64, device="cuda")
                hhg.hhg_residual_noalloc(s.handle, 4, op, u, f, r, norm2)
                torch.cuda.synchronize()
                a, b = r.cpu().numpy(), r_ref.cpu().numpy()
                assert np.linalg.norm(a - b) <= TOL * np.linalg.norm(b), (call, op)
                assert abs(np.sqrt(norm2.item()) - nrm_ref) <= TOL * nrm_ref, (call, op)


def test_noalloc_residual_allocates_nothing():
    """After a first call (which looks up the fixed array's device address),
    further calls leave the device's free memory unchanged."""
    with hhg.Shell(0.55, 1.0, 0, 1, 4) as s:
        s.fit(2, 2)
        n, _ = s.num_nodes()
        u = torch.from_numpy(synthetic.uniform(n, 1)).cuda()
        f = torch.from_numpy(synthetic.uniform(n, 0)).cuda()
        r = torch.empty_like(u)
        norm2 = torch.empty(1, dtype=torch.float64, device="cuda")
        for op in (hhg.HHG_OP_LSQP, hhg.HHG_OP_IFEM):
            hhg.hhg_residual_noalloc(s.handle, 4, op, u, f, r, norm2)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        for _ in range(5):
            for op in (hhg.HHG_OP_LSQP, hhg.HHG_OP_IFEM):
                hhg.hhg_residual_noalloc(s.handle, 4, op, u, f, r, norm2)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0


def test_noalloc_rejects_host_pointers_and_oversized_levels():
    with hhg.Shell(0.55, 1.0, 0, 1, 3) as s:
        n, _ = s.num_nodes()
        u = np.zeros(n)
        norm2 = torch.zeros(1, dtype=torch.float64, device="cuda")
        # the C side rejects host addresses (passed raw, past the binding's checks)
        with pytest.raises(hhg.HHGError) as e:
            hhg.hhg_residual_noalloc(s.handle, 3, hhg.HHG_OP_IFEM, u.ctypes.data, u.ctypes.data, u.ctypes.data,
                                     norm2)
        assert e.value.status == hhg.Status.EINVAL
        # the binding rejects what the C side cannot see: host arrays, wrong
        # type or device, too few values
        d = torch.zeros(n, dtype=torch.float64, device="cuda")
        bad = [
            (u, d, d, norm2),
            (d.float(), d, d, norm2),
            (d, d[: n - 1], d, norm2),
            (d, d, d.cpu(), norm2),
            (d, d, d, torch.zeros(0, dtype=torch.float64, device="cuda")),
            (d, d, d, torch.zeros(1, dtype=torch.float32, device="cuda")),
        ]
        for args in bad:
            with pytest.raises(ValueError):
                hhg.hhg_residual_noalloc(s.handle, 3, hhg.HHG_OP_IFEM, *args)
    # 30720 macro cells need more partial slots than the fixed array holds
    with hhg.Shell(0.55, 1.0, 3, 8, 2) as s:
        n, _ = s.num_nodes()
        u = torch.zeros(n, dtype=torch.float64, device="cuda")
        r = torch.empty_like(u)
        with pytest.raises(hhg.HHGError) as e:
            hhg.hhg_residual_noalloc(s.handle, 2, hhg.HHG_OP_IFEM, u, u, r, norm2)
        assert e.value.status == hhg.Status.EINVAL and "HHG_NOALLOC_SCRATCH" in str(e.value)
