"""The hand-written arithmetic helpers of the surrogate kernels against the
operations they replace, on random operands plus edge cases.

* FP32 divide of the staged FP32 smoother (reciprocal estimate and one
  Newton-Raphson step) vs the correctly rounded IEEE FP32 quotient (NumPy):
  at most 2 ulp, on 2^20 operand pairs over a wide exponent range and
  denominators next to powers of two.
* 2^E / W on the integer pipe (the FP64 surrogate's centre reciprocal: an
  FP32 estimate refined by two fixed-point Newton-Raphson steps) vs the
  exact rational value: at most 2 ulp, on 2^16 integers of 2 to 63 bits,
  both signs, powers of two and their neighbours, and the int64 extremes.
* W 2^-E on the integer pipe (the FP64 surrogate's weights) vs the exact
  value: truncated toward zero, within 1 ulp, 0 for W = 0.
The exact values are Python fractions."""
from fractions import Fraction

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1608_06473_gb300 as hhg  # noqa: E402


def run(which, a, b, out_dtype):
    at = torch.from_numpy(np.ascontiguousarray(a)).cuda()
    bt = torch.from_numpy(np.ascontiguousarray(b)).cuda()
    ot = torch.empty(len(a), dtype=out_dtype, device="cuda")
    hhg.hhg_check_arith(which, at, bt, ot, len(a))
    torch.cuda.synchronize()
    return ot.cpu().numpy()


def test_div_nr32_within_2_ulp():
    n_ = 1 << 20
    rng = np.random.Generator(np.random.PCG64(902))
    sign = lambda m: rng.choice([-1.0, 1.0], m)
    n = (sign(n_) * np.ldexp(rng.uniform(1.0, 2.0, n_), rng.integers(-60, 60, n_))).astype(np.float32)
    d = (sign(n_) * np.ldexp(rng.uniform(1.0, 2.0, n_), rng.integers(-60, 60, n_))).astype(np.float32)
    k = rng.integers(-60, 60, 2048)
    d = np.concatenate([d, np.ldexp(1.0, k).astype(np.float32),
                        np.ldexp(np.float64(np.nextafter(np.float32(2.0), np.float32(0.0))), k).astype(np.float32)])
    n = np.concatenate([n, np.resize(np.array([1.0, -3.0, 0.1, 0.0], dtype=np.float32), 4096)])
    got = run(0, n, d, torch.float32)
    ref = n / d
    assert ref.dtype == np.float32
    ulp = np.spacing(np.abs(ref)).astype(np.float64)
    err = np.abs(got.astype(np.float64) - ref.astype(np.float64))
    assert np.all(err[ref == 0] == 0)
    assert (err[ref != 0] / ulp[ref != 0]).max() <= 2.0


def _int_operands(rng, n):
    bits = rng.integers(1, 63, n)
    W = (rng.integers(1, 1 << 62, n, dtype=np.int64) >> (62 - bits)) | 1
    W = W * rng.choice([-1, 1], n)
    edge = np.array([1, -1, 2, 3, 1 << 62, -(1 << 62), (1 << 62) + 1, (1 << 62) - 1, 1 << 40, (1 << 40) - 1,
                     np.iinfo(np.int64).max, -np.iinfo(np.int64).max, (1 << 53) + 1, 7], dtype=np.int64)
    W = np.concatenate([W, edge]).astype(np.int64)
    E = rng.integers(-40, 120, len(W)).astype(np.int32)
    return W, E


def test_rcp_i64_scaled_within_2_ulp_of_exact():
    rng = np.random.Generator(np.random.PCG64(903))
    W, E = _int_operands(rng, 1 << 16)
    got = run(1, W, E, torch.float64)
    worst = 0.0
    for w, e, g in zip(W.tolist(), E.tolist(), got.tolist()):
        ex = Fraction(2) ** e / w
        worst = max(worst, float(abs(Fraction(g) - ex) / Fraction(float(np.spacing(abs(float(ex)))))))
    assert worst <= 2.0, worst


def test_i64_to_f64_scaled_truncates_within_1_ulp():
    rng = np.random.Generator(np.random.PCG64(904))
    W, E = _int_operands(rng, 1 << 16)
    W[:5] = 0
    got = run(2, W, E, torch.float64)
    for w, e, g in zip(W.tolist(), E.tolist(), got.tolist()):
        if w == 0:
            assert g == 0.0
            continue
        ex = Fraction(w) / Fraction(2) ** e
        assert abs(Fraction(g)) <= abs(ex)          # truncated toward zero
        assert abs(Fraction(g) - ex) <= Fraction(float(np.spacing(abs(float(ex)))))
        assert (g < 0) == (w < 0)
