"""Serving: requests of mixed geometry, level and right-hand-side count run
concurrently on the server's slots (own host thread and CUDA stream each)
over resident hierarchies.  Every request's result must be the same alone
and in the mix: to 1e-12 relative in FP64 (the same arithmetic on the same
hierarchy contents) and to 1e-6 relative in mixed precision (both reach the
1e-8 residual; the FP32 smoother configuration is chosen per hierarchy by
timing, which may change the rounding).  Also: every result reaches the
tolerance and equals a direct hhg_vcycle solve; a hierarchy is reused by a
later request of the same key; a request that cannot fit the budget fails
with HHG_ENOMEM instead of waiting forever."""
import numpy as np
import pytest

import synthetic

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1608_06473_gb300 as hhg  # noqa: E402

# (r_inner, L, nrhs) on the 60-macro shell
MIX = [(0.45, 4, 2), (0.55, 3, 1), (0.45, 4, 1), (0.6, 4, 3), (0.55, 3, 2), (0.6, 5, 1), (0.45, 3, 1), (0.55, 4, 2)]


def rhs(k, r_inner, L, nrhs):
    n, _ = hhg.hhg_problem_nodes(r_inner, 1.0, 0, 1, L)
    return np.stack([synthetic.uniform(n, 500 + 16 * k + b) for b in range(nrhs)])


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("dtype,tol", [(hhg.HHG_F64, 1e-12), (hhg.HHG_F32, 1e-6)])
def test_mix_equals_alone(dtype, tol):
    fs = [rhs(k, ri, L, nr) for k, (ri, L, nr) in enumerate(MIX)]
    with hhg.Server(max_inflight=3, dtype=dtype) as srv:
        tickets = [srv.submit(f, r_inner=ri, L=L) for f, (ri, L, _) in zip(fs, MIX)]
        mix = [srv.wait(t) for t in tickets]
        stats = srv.stats()
    assert stats["built"] <= len(MIX)
    with hhg.Server(max_inflight=1, dtype=dtype) as srv:
        alone = []
        for f, (ri, L, _) in zip(fs, MIX):
            alone.append(srv.wait(srv.submit(f, r_inner=ri, L=L)))
    for (um, rm, im), (ua, ra, ia) in zip(mix, alone):
        assert np.all(rm <= 1e-8) and np.all(ra <= 1e-8)
        assert rel(um, ua) <= tol
        assert im["t_submit"] <= im["t_start"] <= im["t_end"]


def test_matches_direct_solve_and_reuses_hierarchies():
    ri, L, nr = 0.5, 4, 2
    f = rhs(99, ri, L, nr)
    with hhg.Server(max_inflight=2, dtype=hhg.HHG_F64) as srv:
        u1, r1, i1 = srv.wait(srv.submit(f, r_inner=ri, L=L))
        u2, r2, i2 = srv.wait(srv.submit(f, r_inner=ri, L=L))
        assert not i1["reused"] and i2["reused"]
        assert srv.stats()["resident"] == 1
    assert rel(u2, u1) == 0.0
    with hhg.Shell(ri, 1.0, 0, 1, L) as s:
        s.fit(2, 2)
        ft = torch.from_numpy(f).cuda()
        ut = torch.zeros_like(ft)
        s.vcycle(ft, ut, nrhs=nr, rtol=1e-8, max_cycles=60)
        torch.cuda.synchronize()
        assert rel(u1, ut.cpu().numpy()) <= 1e-12


def test_request_that_cannot_fit_fails():
    f = rhs(7, 0.55, 4, 1)
    with hhg.Server(hbm_budget_bytes=1 << 20, max_inflight=1, dtype=hhg.HHG_F64) as srv:
        t = srv.submit(f, r_inner=0.55, L=4)
        with pytest.raises(hhg.HHGError) as e:
            srv.wait(t)
        assert e.value.status == hhg.Status.ENOMEM


@pytest.mark.parametrize("dtype,tol", [(hhg.HHG_F64, 1e-10), (hhg.HHG_F32, 1e-6)])
def test_continuous_batching_equals_alone(dtype, tol):
    """Continuous batching (max_batch_rhs): requests of one key queued while
    its hierarchy is busy are merged into one batched solve, and every
    right-hand side is stopped at its own convergence, so each request gets
    the result and cycle count of the same request solved alone with the same
    setting (to the batched kernels' rounding: 1e-10 in FP64, the
    mixed-precision bar in FP32)."""
    ri, L = 0.55, 4
    fs = [rhs(200 + k, ri, L, nr) for k, nr in enumerate([1, 2, 1, 3, 1, 2])]
    with hhg.Server(max_inflight=1, dtype=dtype, max_batch_rhs=8) as srv:
        tickets = [srv.submit(f, r_inner=ri, L=L) for f in fs]
        merged = [srv.wait(t) for t in tickets]
    with hhg.Server(max_inflight=1, dtype=dtype, max_batch_rhs=8) as srv:
        alone = [srv.wait(srv.submit(f, r_inner=ri, L=L)) for f in fs]
    assert any(im["batch_rhs"] > len(f) for f, (_, _, im) in zip(fs, merged))
    for f, (um, rm, im), (ua, ra, ia) in zip(fs, merged, alone):
        assert ia["batch_rhs"] == len(f) and im["batch_rhs"] >= len(f)
        assert np.all(rm <= 1e-8) and np.all(ra <= 1e-8)
        if dtype == hhg.HHG_F64:
            assert im["cycles"] == ia["cycles"]
        assert rel(um, ua) <= tol


def test_budget_evicts_least_recently_used():
    """Under an HBM budget that holds two hierarchies of a level but not
    three, a request of a third key evicts the least recently used idle
    hierarchy (one, not all), and a later request of the evicted key
    rebuilds it; results equal those of an unbudgeted server (FP64: the same
    arithmetic on a rebuilt hierarchy)."""
    keys = [(0.45, 4), (0.55, 4), (0.65, 4), (0.45, 4)]
    fs = [rhs(300 + k, ri, L, 1) for k, (ri, L) in enumerate(keys)]
    with hhg.Server(max_inflight=1, dtype=hhg.HHG_F64) as srv:
        ref = [srv.wait(srv.submit(f, r_inner=ri, L=L)) for f, (ri, L) in zip(fs, keys)]
        st0 = srv.stats()
    assert st0["built"] == 3 and st0["evicted"] == 0
    per = st0["bytes"] / 3
    vec = 2 * fs[0].size * 8
    # room for two resident hierarchies and a few request vectors, not for a third
    with hhg.Server(hbm_budget_bytes=int(2 * per) + 4 * vec, max_inflight=1, dtype=hhg.HHG_F64) as srv:
        got = []
        for f, (ri, L) in zip(fs, keys):
            got.append(srv.wait(srv.submit(f, r_inner=ri, L=L)))
            assert srv.stats()["resident"] <= 2
        st = srv.stats()
    # key 0 evicted by key 2, then key 1 by the rebuild of key 0
    assert st["evicted"] == 2 and st["built"] == 4
    assert [i["reused"] for _, _, i in got] == [0, 0, 0, 0]
    for (ug, rg, _), (ur, rr, _) in zip(got, ref):
        assert np.all(rg <= 1e-8)
        assert rel(ug, ur) <= 1e-12
