"""Seeded query streams: node pairs, error targets, per-query RNG seeds, arrivals.

Query pairs are drawn uniformly among ordered pairs with s != t, as in the
paper's query sets (Section 4.1).
"""

from __future__ import annotations

import numpy as np


def uniform_pairs(n: int, count: int, seed: int) -> tuple[np.ndarray, np.ndarray]:
    rng = np.random.default_rng(seed)
    s = rng.integers(0, n, size=count, dtype=np.int64)
    t = rng.integers(0, n - 1, size=count, dtype=np.int64)
    t = t + (t >= s)
    return s, t


def eps_uniform(count: int, lo: float, hi: float, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=count)


def eps_choice(count: int, choices, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.choice(np.asarray(choices, dtype=np.float64), size=count)


def query_seeds(count: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.integers(0, 2**63 - 1, size=count, dtype=np.int64).astype(np.uint64)


def poisson_arrivals(count: int, rate_per_s: float, seed: int) -> np.ndarray:
    """Arrival times (seconds) of a Poisson process with the given rate."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_per_s, size=count))
