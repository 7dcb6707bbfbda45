"""Seeded synthetic inputs (no arithmetic of the method itself).

Shared by the benchmark and the tests: parameter sets and path counts of the
batched sweep workload, drawn with numpy's PCG64 from a fixed seed.
"""
from __future__ import annotations

import numpy as np


def sweep_sets(n_sets: int = 4096, seed: int = 0):
    """CIR parameter sets of the batched sweep: kappa ~ U(0.1, 2),
    theta ~ U(0.01, 0.1), sigma ~ U(0.1, 0.5), X0 = theta, T = 1, and a base
    path count n_s log-uniform on [1e3, 1e6]."""
    rng = np.random.default_rng(seed)
    kappa = rng.uniform(0.1, 2.0, n_sets)
    theta = rng.uniform(0.01, 0.1, n_sets)
    sigma = rng.uniform(0.1, 0.5, n_sets)
    n_base = np.floor(10.0 ** rng.uniform(3.0, 6.0, n_sets)).astype(np.int64)
    return {"kappa": kappa, "theta": theta, "sigma": sigma, "X0": theta.copy(), "T": 1.0,
            "n_base": n_base}


def sweep_counts(n_base: np.ndarray, levels: int = 8, corr_ratio: int = 256, floor: int = 1000):
    """Fixed-work path counts per (set, level): the approximate two-way term
    gets max(floor, n_s 2^-l) paths and the four-way correction 1/corr_ratio of
    that (at least 256)."""
    n2 = np.maximum(floor, n_base[:, None] >> np.arange(levels)[None, :])
    n4 = np.maximum(256, n2 // corr_ratio)
    return n2, n4
