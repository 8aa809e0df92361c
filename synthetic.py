"""Seeded synthetic inputs shared by the tests, the bench and the oracle.

Holds no arithmetic of the method: only random vectors and index samples,
generated on the host with NumPy's PCG64 so that the CUDA path and the CPU
oracle receive bit-identical inputs.  Vectors cover all canonical nodes;
entries at Dirichlet nodes are ignored by both sides.

Seeds: right-hand side f -> 0, iterate u for operator timing -> 1, right-hand
side number b of a batch -> 100 + b.
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
