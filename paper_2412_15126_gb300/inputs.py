"""Seeded synthetic workloads (Sec. 6.1: values drawn uniformly at random in a
bounded interval).  Used by the tests, the benchmark and the smoke check for
both the CUDA path and the oracle; holds none of the method's arithmetic.

* ``gap_vector``: N values in [0, 1) whose pairwise distances are >= gap, drawn
  uniformly over such configurations (N uniforms on [0, 1 - (N-1) gap], sorted,
  the i-th shifted by i*gap, then a seeded random permutation).
* ``grid_vector``: N values on a `levels`-point grid in [0, 1), so ties occur.
* ``batch_lengths``: the mixed-length batch of rank queries.
"""
from __future__ import annotations

import numpy as np


def gap_vector(N: int, gap: float, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    span = 1.0 - (N - 1) * gap
    if span <= 0:
        raise ValueError("gap too large for N values in [0, 1)")
    u = np.sort(rng.uniform(0.0, span, N)) + np.arange(N) * gap
    return rng.permutation(u)


def grid_vector(N: int, levels: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.integers(0, levels, N) / float(levels)


def batch_lengths(count: int, choices=(16, 32, 64, 128), seed: int = 4) -> list:
    rng = np.random.default_rng(seed)
    return [int(x) for x in rng.choice(np.asarray(choices), size=count)]
