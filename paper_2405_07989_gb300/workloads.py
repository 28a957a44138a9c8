"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module only draws inputs; it holds none of the method's arithmetic.  The
paper measures on printed inputs (Table 1, Sec. 5.2) and no dataset, so every
workload here is either one of those printed inputs or a seeded draw with the
shapes the benchmark configurations name.
"""
from __future__ import annotations

import numpy as np

# Tiny query, plain method: the oracle finishes it in well under a second.
CONFIG1 = (500, (5, 7, 11, 13))
# Single large query: about 7.2e7 factorizations, 1.73 GB of int32 rows.
CONFIG2 = (3000, (11, 13, 17, 19, 23, 29))

# Table 1 generator families (Sec. 5.2): "...,40" means (13,37,38,40), etc.
TABLE1_GENS = {
    3: (13, 37, 38),
    4: (13, 37, 38, 40),
    5: (13, 37, 38, 40, 41),
    6: (13, 37, 38, 40, 41, 42),
    7: (13, 37, 38, 40, 41, 42, 43),
}


def config3(seed: int = 0, n: int = 40000):
    """Count-only heavy query: 8 distinct generators uniform in [50, 200]."""
    rng = np.random.default_rng(seed)
    g = rng.choice(np.arange(50, 201), 8, replace=False)
    return n, tuple(int(x) for x in g)


def config4(seed: int = 0, nq: int = 4096, n_max: int = 5000):
    """Batched queries: d uniform in [3, 8], distinct generators uniform in
    [5, 100], n uniform in [100, n_max]."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(nq):
        d = int(rng.integers(3, 9))
        g = rng.choice(np.arange(5, 101), d, replace=False)
        n = int(rng.integers(100, n_max + 1))
        out.append((n, tuple(int(x) for x in g)))
    return out


def config5(seed: int = 0, nreq: int = 2000, rate: float = 1000.0, n_max: int = 20000):
    """Serving requests: queries drawn like the batched ones with n up to
    n_max, Poisson arrivals at `rate` per second, and an operation drawn as
    count / length-stats / enumerate with probabilities 0.8 / 0.15 / 0.05.
    Returns a list of (arrival_seconds, op, n, gens)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for _ in range(nreq):
        d = int(rng.integers(3, 9))
        g = rng.choice(np.arange(5, 101), d, replace=False)
        n = int(rng.integers(100, n_max + 1))
        t += float(rng.exponential(1.0 / rate))
        op = int(rng.choice(3, p=[0.8, 0.15, 0.05]))
        out.append((t, op, n, tuple(int(x) for x in g)))
    return out


def random_small(seed: int, count: int, d_max: int = 4, n_max: int = 60, g_max: int = 12,
                 repeats: bool = True):
    """Tiny random queries for brute-force comparisons (repeated generators allowed)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        d = int(rng.integers(1, d_max + 1))
        if repeats:
            g = rng.integers(1, g_max + 1, size=d)
        else:
            g = rng.choice(np.arange(1, g_max + 1), min(d, g_max), replace=False)
        n = int(rng.integers(0, n_max + 1))
        out.append((n, tuple(int(x) for x in g)))
    return out


def random_medium(seed: int, count: int, d_lo: int = 1, d_hi: int = 9, g_lo: int = 2,
                  g_hi: int = 60, n_lo: int = 0, n_hi: int = 400):
    """Random queries of moderate size for parity tests (several tiles, ragged)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        d = int(rng.integers(d_lo, d_hi))
        g = rng.integers(g_lo, g_hi + 1, size=d)
        n = int(rng.integers(n_lo, n_hi + 1))
        out.append((n, tuple(int(x) for x in g)))
    return out
