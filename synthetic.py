"""Seeded synthetic inputs shared by the tests, the bench and the oracle.

Holds no arithmetic of the method: only random vectors and index samples,
generated on the host with NumPy's PCG64 so that the CUDA path and the CPU
oracle receive bit-identical inputs.  Vectors cover all canonical nodes;
entries at Dirichlet nodes are ignored by both sides.

Seeds: right-hand side f -> 0, iterate u for operator timing -> 1, right-hand
side number b of a batch -> 100 + b.

Besides the random vectors it holds the analytic problem data of the paper's
accuracy study (Sec. 4): the exact solution and its right-hand side, as
functions of position.  That is input data of the study, not arithmetic of
the method.
"""
from __future__ import annotations

import numpy as np

SEED_F = 0
SEED_U = 1
SEED_BATCH0 = 100


def uniform(n: int, seed: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """n values uniform in [lo, hi), float64."""
    return np.random.Generator(np.random.PCG64(seed)).uniform(lo, hi, n)


def gaussian(n: int, seed: int, sigma: float = 1.0) -> np.ndarray:
    """n values N(0, sigma^2), float64."""
    return np.random.Generator(np.random.PCG64(seed)).normal(0.0, sigma, n)


def batch(n: int, nrhs: int, dist: str = "uniform") -> np.ndarray:
    """nrhs vectors (rows) with seeds 100 + b."""
    gen = uniform if dist == "uniform" else gaussian
    return np.stack([gen(n, SEED_BATCH0 + b) for b in range(nrhs)])


def sample(n: int, k: int, seed: int) -> np.ndarray:
    """k distinct sorted integers from range(n)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.sort(rng.choice(n, size=min(k, n), replace=False))


def manufactured(X, r1: float, r2: float, xp=np):
    """Exact solution u = (r - r1)(r - r2) sin(10x) sin(4y) sin(7z) of the
    accuracy study (Sec. 4, with r = |x|) and f = -Laplace(u), at the rows of
    X (n, 3).  With g(r) = (r - r1)(r - r2) and S the sine product:
    Laplace(g S) = (g'' + 2 g'/r) S + 2 (g'/r) (x . grad S) + g Laplace(S),
    g' = 2r - r1 - r2, g'' = 2, Laplace(S) = -(100 + 16 + 49) S.  Works on
    NumPy arrays (xp = numpy) and on torch tensors (xp = torch)."""
    x, y, z = X[:, 0], X[:, 1], X[:, 2]
    r = xp.sqrt(x * x + y * y + z * z)
    sx, sy, sz = xp.sin(10 * x), xp.sin(4 * y), xp.sin(7 * z)
    S = sx * sy * sz
    g = (r - r1) * (r - r2)
    gp = 2 * r - (r1 + r2)
    x_grad_S = (10 * x * xp.cos(10 * x) * sy * sz + 4 * y * sx * xp.cos(4 * y) * sz
                + 7 * z * sx * sy * xp.cos(7 * z))
    lap = (2 + 2 * gp / r) * S + 2 * (gp / r) * x_grad_S - 165 * g * S
    return g * S, -lap
