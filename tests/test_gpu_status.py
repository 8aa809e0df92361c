"""Failure statuses of the V-cycle driver, made on the host side of the C ABI
(Sec. 4's stopping rule: cycles stop at ||f - L u|| <= rtol ||f - L u_0||).

* A tolerance no cycle count can reach within max_cycles gives HHG_ENOCONV,
  with the relative residual actually reached and the cycles run filled in.
* A NaN or an Inf written into the host right-hand side before the call
  gives HHG_EDIVERGED (the initial residual norm is not finite), and the
  shell stays usable for the next, finite solve.
Nothing here faults, traps or hangs the GPU: the bad values are ordinary
floating-point data, and the checks are host-side reads of residual norms."""
import numpy as np
import pytest

import synthetic

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1608_06473_gb300 as hhg  # noqa: E402


@pytest.fixture(scope="module")
def c1():
    with hhg.Shell(0.55, 1.0, 0, 1, 4) as s:
        s.fit(2, 2)
        yield s


@pytest.mark.parametrize("dtype", [hhg.HHG_F64, hhg.HHG_F32])
def test_enoconv_reports_reached_relres(c1, dtype):
    s = c1
    n, _ = s.num_nodes()
    f = torch.from_numpy(synthetic.uniform(n, synthetic.SEED_F)).cuda()
    u = torch.zeros_like(f)
    rel, cycles, st = s.vcycle(f, u, max_cycles=1, rtol=1e-30, dtype=dtype, raise_on_noconv=False)
    assert st == hhg.HHG_ENOCONV
    assert cycles == 1
    # one V(3,3) cycle reduces the residual by a factor well below 1, and
    # the value is the one reached, not a placeholder
    assert 0.0 < rel[0] < 0.5
    with pytest.raises(hhg.HHGError) as e:
        s.vcycle(f, torch.zeros_like(f), max_cycles=1, rtol=1e-30, dtype=dtype)
    assert e.value.status == hhg.Status.ENOCONV
    # the same cycle, allowed to converge, meets the tolerance
    rel2, cycles2, st2 = s.vcycle(f, torch.zeros_like(f), rtol=1e-8, dtype=dtype)
    assert st2 == hhg.HHG_OK and rel2[0] <= 1e-8 and cycles2 > 1


@pytest.mark.parametrize("bad", [np.nan, np.inf, -np.inf])
@pytest.mark.parametrize("dtype", [hhg.HHG_F64, hhg.HHG_F32])
def test_ediverged_on_non_finite_host_rhs(c1, bad, dtype):
    s = c1
    n, _ = s.num_nodes()
    f = synthetic.uniform(n, synthetic.SEED_F)
    f[n - 7] = bad            # a cell-interior node (canonical order ends with the cells)
    u = np.zeros(n)
    with pytest.raises(hhg.HHGError) as e:
        s.vcycle(f, u, dtype=dtype)
    assert e.value.status == hhg.Status.EDIVERGED
    # the shell still solves a finite problem afterwards
    f[n - 7] = 0.5
    u = np.zeros(n)
    rel, _, st = s.vcycle(f, u, dtype=dtype)
    assert st == hhg.HHG_OK and rel[0] <= 1e-8 and np.all(np.isfinite(u))
