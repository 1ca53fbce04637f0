"""Seeded random population states for single-cell unit tests.

States are ``w_i * (1 + amplitude * r_i)`` with ``r_i`` uniform in [-1, 1]:
positive, near the rest state, with random density, momentum and stress.
The caller passes the lattice weights (from whichever implementation it
tests against); nothing of the collision scheme is evaluated here.
"""

from __future__ import annotations

import numpy as np


def random_populations(seed: int, n: int, weights, amplitude: float = 0.1) -> np.ndarray:
    w = np.asarray(weights, dtype=np.float64)
    rng = np.random.Generator(np.random.PCG64(seed))
    r = rng.uniform(-1.0, 1.0, size=(n, w.size))
    return w[None, :] * (1.0 + amplitude * r)
