"""Seeded synthetic inputs shared by the CUDA path's tests/benchmark and the oracle.

This module draws random numbers only; it holds none of the likelihood's
arithmetic.  Recipes (the paper's workloads are synthetic Matérn fields on the
unit square, Section III, Examples 1-2):

* locations: an m x m grid on [0, 1]^2 with every point jittered uniformly by
  +-0.4 of a cell, s = ((i + 0.5 + U) / m, (j + 0.5 + V) / m), U, V ~ U(-0.4, 0.4),
  x index fastest (the order of R's expand.grid used in Section III);
  minimum spacing is then >= 0.2 / m.
* eps ~ N(0, 1) i.i.d.; an exact realisation is Z = L eps with L L^T = Sigma(theta0)
  (Section III, Example 1), formed by the caller.
* theta perturbations: theta0 * exp(0.2 u), u ~ U(-1, 1)^3, clipped to bounds.
* replicate sizes: n_i = m_i^2 with m_i ~ U{20..80}.

Seeds: locations use ``seed``, eps ``seed + 1``, theta perturbations ``seed + 2``
(numpy PCG64 via default_rng).
"""
from __future__ import annotations

import numpy as np

# sigma^2, beta, nu bounds of the bounded MLE search
THETA_LOWER = np.array([0.01, 0.01, 0.1])
THETA_UPPER = np.array([5.0, 2.0, 2.0])


def jittered_grid(m: int, seed: int, jitter: float = 0.4) -> np.ndarray:
    """n = m*m locations, shape (n, 2), float64, x index fastest."""
    rng = np.random.default_rng(seed)
    u = rng.uniform(-jitter, jitter, size=(m * m, 2))
    jj, ii = np.meshgrid(np.arange(m), np.arange(m), indexing="ij")  # jj: y index, ii: x index
    base = np.stack([ii.ravel(), jj.ravel()], axis=1).astype(np.float64)
    return np.ascontiguousarray((base + 0.5 + u) / m)


def normals(n: int, seed: int) -> np.ndarray:
    return np.random.default_rng(seed + 1).standard_normal(n)


def theta_perturbations(theta0, count: int, seed: int, lower=THETA_LOWER, upper=THETA_UPPER) -> np.ndarray:
    rng = np.random.default_rng(seed + 2)
    u = rng.uniform(-1.0, 1.0, size=(count, 3))
    th = np.asarray(theta0, dtype=np.float64)[None, :] * np.exp(0.2 * u)
    return np.clip(th, lower, upper)


def replicate_sides(count: int, seed: int, lo: int = 20, hi: int = 80) -> np.ndarray:
    """Grid sides m_i ~ U{lo..hi}; replicate i has n_i = m_i^2 locations."""
    return np.random.default_rng(seed).integers(lo, hi + 1, size=count)


def uniform_square(n: int, seed: int) -> np.ndarray:
    """n i.i.d. uniform locations on [0, 1]^2 (simulate_data_exact's design)."""
    return np.ascontiguousarray(np.random.default_rng(seed).uniform(0.0, 1.0, size=(n, 2)))
