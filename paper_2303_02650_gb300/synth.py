"""Seeded synthetic inputs shared by the tests and the benchmark.

This module only draws numbers: instance sizes, container radii and arbitrary
test layouts.  It holds none of the descent's arithmetic (the method's own
random initial layout is drawn on each side from Philox4x32-10).

Workloads (the paper's instances are just values of n, Sec. 6.1):
  * single_instance(n, u): R = sqrt(n / u)
  * batch_manifest(num, seed): n ~ U{300..1000}, u ~ U[0.80, 0.84], R = sqrt(n / u)
  * random_layout(n, R, seed): centres uniform in the square [-R, R]^2
  * hex_patch(rings, spacing): a hexagonal patch of 3 r (r + 1) + 1 centres
"""
from __future__ import annotations

import numpy as np


def radius(n: int, u: float) -> float:
    """Container radius for n unit circles at density u = n / R^2."""
    return float(np.sqrt(n / u))


def batch_manifest(num: int = 4096, seed: int = 2303, n_lo: int = 300, n_hi: int = 1000,
                   u_lo: float = 0.80, u_hi: float = 0.84):
    """Independent instances of uneven size: returns (n int32[num], R float64[num])."""
    g = np.random.Generator(np.random.Philox(seed))
    n = g.integers(n_lo, n_hi + 1, size=num).astype(np.int32)
    u = g.uniform(u_lo, u_hi, size=num)
    R = np.sqrt(n / u)
    return n, R


def random_layout(n: int, R: float, seed: int, spread: float = 1.0) -> np.ndarray:
    """Arbitrary test layout: centres uniform in [-spread R, spread R]^2, float64 [n, 2]."""
    g = np.random.Generator(np.random.Philox(seed))
    return g.uniform(-spread * R, spread * R, size=(n, 2))


def hex_patch(rings: int, spacing: float) -> np.ndarray:
    """Centres of a hexagonal patch with the given number of rings around the origin."""
    pts = []
    for q in range(-rings, rings + 1):
        for r in range(max(-rings, -q - rings), min(rings, -q + rings) + 1):
            pts.append((spacing * (q + 0.5 * r), spacing * (np.sqrt(3.0) / 2.0) * r))
    return np.asarray(pts, dtype=np.float64)
