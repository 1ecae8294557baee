"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle
comparisons.  Holds none of the method's arithmetic: only input
distributions over {0,1}^n, deletion-probability grids and random
coordinates.

Input strings are integers with x_0 as the most significant of n bits.
"""
from __future__ import annotations

import numpy as np


def uniform_p(n: int, nd: int = 1) -> np.ndarray:
    """X^(0) of every configuration: uniform over {0,1}^n."""
    return np.full((nd, 1 << n), 1.0 / (1 << n))


def _rev(x: np.ndarray, n: int) -> np.ndarray:
    r = np.zeros_like(x)
    for i in range(n):
        r |= ((x >> i) & 1) << (n - 1 - i)
    return r


def orbit_invariant_dirichlet(n: int, seed: int = 0, nd: int = 1) -> np.ndarray:
    """Dirichlet(1) draw (numpy default_rng(seed)) averaged over the
    complement/reversal orbit of each input, so that it is orbit-invariant
    like every BA iterate from a uniform start."""
    rng = np.random.default_rng(seed)
    out = np.zeros((nd, 1 << n))
    x = np.arange(1 << n, dtype=np.int64)
    full = (1 << n) - 1
    rx = _rev(x, n)
    for z in range(nd):
        p = rng.dirichlet(np.ones(1 << n))
        ps = (p[x] + p[x ^ full] + p[rx] + p[rx ^ full]) / 4.0
        out[z] = ps / ps.sum()
    return out


def batched_d_grid() -> dict:
    """Batched sweep workload: n=22 with 32 values of d evenly spaced over
    [0.05, 0.95], and n in {14,16,18,20} with 8 values each in [0.6, 0.95]."""
    g = {22: [0.05 + 0.9 * i / 31 for i in range(32)]}
    mixed = [0.60 + 0.05 * i for i in range(8)]
    for n in (14, 16, 18, 20):
        g[n] = list(mixed)
    return g


LARGE_SWEEP_D = [0.64, 0.70, 0.75, 0.80, 0.85, 0.90, 0.95]


def random_codes(n: int, count: int, seed: int = 0) -> np.ndarray:
    """Output codes (1<<k)|y spread over every length k = 0..n."""
    rng = np.random.default_rng(seed)
    ks = rng.integers(0, n + 1, size=count)
    ys = np.array([rng.integers(0, 1 << k) if k > 0 else 0 for k in ks], dtype=np.int64)
    return (np.int64(1) << ks.astype(np.int64)) | ys


def random_inputs(n: int, count: int, seed: int = 0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.integers(0, 1 << n, size=count, dtype=np.int64)


def fd_coordinates(num: int, count: int, seed: int = 0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.choice(num, size=min(count, num), replace=False)
