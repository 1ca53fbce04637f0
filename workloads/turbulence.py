"""Random-Fourier-mode table for the synthetic turbulent inflow.

The inflow perturbation is a frozen, divergence-free sum of ``n_modes``
Fourier modes ``a_m cos(k_m . x') + b_m sin(k_m . x')``; this module only
draws the table ``(k_m, a_m, b_m)`` from a seeded PCG64 stream.  Wave
numbers are log-uniform in magnitude between ``2 pi / length`` and
``2 pi / 4`` with isotropic directions; ``a_m`` and ``b_m`` are projected
orthogonal to ``k_m`` (divergence-free) and share the energy equally, scaled
so that the mean per-component rms of the perturbation is
``intensity * u_mean``.
"""

from __future__ import annotations

import numpy as np


def inflow_plane(modes, shape, flow_axis: int, u_mean: float, t: int) -> np.ndarray:
    """The synthetic inflow on the inlet plane (flow-axis coordinate 0) at
    step t, as input data for a caller-supplied inflow:
    u = u_mean a + sum_m a_m cos(k_m . x') + b_m sin(k_m . x'), x' = x - u_mean t a.
    shape = (nx, ny, nz); returns float64 (3, n_c, n_b), (b, c) = the axes
    after flow_axis in cyclic order, b fastest."""
    b, c = (flow_axis + 1) % 3, (flow_axis + 2) % 3
    nb, nc = shape[b], shape[c]
    X = np.zeros((3, nc, nb))
    X[b] = np.arange(nb)[None, :]
    X[c] = np.arange(nc)[:, None]
    X[flow_axis] = -u_mean * t
    u = np.zeros((3, nc, nb))
    u[flow_axis] = u_mean
    if modes is not None:
        for m in np.asarray(modes, dtype=np.float64).reshape(-1, 9):
            ph = m[0] * X[0] + m[1] * X[1] + m[2] * X[2]
            cs, sn = np.cos(ph), np.sin(ph)
            for k in range(3):
                u[k] += m[3 + k] * cs + m[6 + k] * sn
    return u


def fourier_modes(seed: int, n_modes: int = 64, length: float = 256.0,
                  u_mean: float = 0.05, intensity: float = 0.05,
                  kmax_wavelength: float = 4.0) -> np.ndarray:
    """Return a float64 array of shape (n_modes, 9): k(3), a(3), b(3)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    kmin = 2.0 * np.pi / length
    kmax = 2.0 * np.pi / kmax_wavelength
    kmag = np.exp(rng.uniform(np.log(kmin), np.log(kmax), n_modes))
    dirs = rng.normal(size=(n_modes, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    k = kmag[:, None] * dirs
    a = rng.normal(size=(n_modes, 3))
    b = rng.normal(size=(n_modes, 3))
    a -= np.sum(a * dirs, axis=1, keepdims=True) * dirs
    b -= np.sum(b * dirs, axis=1, keepdims=True) * dirs
    e = np.sum(a * a + b * b, axis=1, keepdims=True)
    # equal energy per mode; mean square per component = sum_m e_m / 6
    target = 6.0 * (intensity * u_mean) ** 2 / n_modes
    a *= np.sqrt(target / e)
    b *= np.sqrt(target / e)
    return np.ascontiguousarray(np.concatenate([k, a, b], axis=1))
