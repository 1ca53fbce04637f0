"""The GPU wall model (FP32 Newton with the exp(-kappa u+)-scaled step) in the
log-law regime, against the same closed forms that pin the oracle
(Sec. 2.2.1): a log-law velocity field u = u_tau/kappa ln(E y u_tau/nu)
around an oblique flat wall (a finite patch of the plane, so that the rotor's
box fits the lattice), with a wall-normal flow added and with a moving wall;
one evaluation from a cold start.  The expected values come from the
prescribed field alone: the sample velocity by a library trilinear
interpolation, u_tau and u+ as brentq roots of the explicit Eq. (spalding),
the strain as the symmetric gradient of the straight profile between the
wall cell and the sample.  FP32 arithmetic (the velocity moment of the stored
equilibrium, the binary32 level set and normal, the Newton iterates) limits
the agreement to ~1e-6; the bound is 2e-5.
"""

import math

import numpy as np
import pytest
from scipy.ndimage import map_coordinates
from scipy.optimize import brentq

from workloads import BladeGrid

pytestmark = pytest.mark.gpu

E, KAPPA = 9.8, 0.41
TAU = 0.50005
NU = (TAU - 0.5) / 3.0
YS = 2.0
UT_STAR = 0.002
SHAPE = (56, 56, 40)
N_HAT = np.array([0.35, 1.0, 0.25]) / np.linalg.norm([0.35, 1.0, 0.25])


def _yplus(up):
    k = KAPPA * up
    return up + (math.exp(k) - 1.0 - k - k * k / 2.0 - k ** 3 / 6.0) / E


def _uplus(yp):
    return brentq(lambda v: _yplus(v) - yp, 1e-9, 80.0, xtol=1e-15, rtol=1e-15)


def _utau(u, y):
    return brentq(lambda ut: _yplus(u / ut) - y * ut / NU, u / 150.0, u, xtol=1e-16, rtol=1e-15)


def _patch_grid(center, p0, half=(9.0, 9.0, 4.0), h=0.5):
    """Blade-frame level set of the plane n.(x - p0) = 0 on a patch of
    half-widths `half` around the rotor centre (frame = lab shifted by the
    centre for a rotor about z at angle 0)."""
    axes = [np.arange(-half[k], half[k] + 1e-9, h) for k in range(3)]
    AA, TT, RR = np.meshgrid(axes[2], axes[1], axes[0], indexing="ij")
    phi = (N_HAT[0] * (RR + center[0] - p0[0]) + N_HAT[1] * (TT + center[1] - p0[1])
           + N_HAT[2] * (AA + center[2] - p0[2]))
    return BladeGrid(sdf=np.ascontiguousarray(phi.astype(np.float32)), origin=(-half[0], -half[1], -half[2]),
                     spacing=h, radius=1.0, hub_radius=0.0, chord_root=1.0, chord_tip=1.0)


def _solid_velocity(omega, c, X, Y, Z):
    X = np.asarray(X, float)
    return np.stack([-omega * (np.asarray(Y, float) - c[1]), omega * (X - c[0]), 0.0 * X])


@pytest.mark.parametrize("case", ["static", "normal_flow", "moving_wall"])
def test_gpu_wall_model_closed_form_log_law(case):
    import torch
    if not torch.cuda.is_available():
        pytest.fail("a CUDA device is required for the gpu-marked tests")
    from paper_2510_13726_b300.build import build
    build()
    import paper_2510_13726_b300 as P
    nx, ny, nz = SHAPE
    center = (27.5, 27.5, 19.5)
    p0 = np.array([27.1, 26.8, 19.2])
    omega = 6e-5 if case == "moving_wall" else 0.0
    u_normal = 0.012 if case == "normal_flow" else 0.0
    t0 = np.cross(N_HAT, [0.0, 0.0, 1.0])
    t0 /= np.linalg.norm(t0)
    lat = P.Lattice(nx, ny, nz, open_boundaries=False, tau_mo=TAU, c_smag=0.1, u_in=0.0, wall_model=True,
                    wm_tol=1e-13, wm_maxit=100, mass_check_every=0)
    lat.add_rotor(_patch_grid(center, p0), center=center, omega=omega, axis=2, n_blades=1, hub_radius=0.0)
    Z, Y, X = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    phi = N_HAT[0] * (X - p0[0]) + N_HAT[1] * (Y - p0[1]) + N_HAT[2] * (Z - p0[2])
    U = np.where(phi > 0.05, UT_STAR / KAPPA * np.log(E * np.maximum(phi, 1e-3) * UT_STAR / NU), 0.0)
    u = _solid_velocity(omega, center, X, Y, Z) + U[None] * t0[:, None, None, None] \
        + u_normal * N_HAT[:, None, None, None]
    u32 = u.astype(np.float32)
    lat.init_fields(torch.ones(nz * ny * nx), torch.tensor(u32.reshape(3, -1)))
    lat.step(1)
    band = lat.rotor_band(0)
    lo = band["lo"]
    flags = band["flags"].cpu().numpy()
    wm = band["wm"].cpu().numpy().astype(np.float64)
    ut = band["utau"].cpu().numpy()
    wall = np.argwhere((flags & 2) > 0)
    # interior of the patch: the level set there is the plane's
    checked = 0
    for bz, by, bx in wall:
        x, y, z = bx + lo[0], by + lo[1], bz + lo[2]
        if max(abs(x - center[0]), abs(y - center[1])) > 6 or abs(z - center[2]) > 2:
            continue
        xs = np.array([x, y, z], float) + YS * N_HAT
        coords = np.array([[xs[2]], [xs[1]], [xs[0]]])
        us = np.array([map_coordinates(u32[k].astype(np.float64), coords, order=1)[0] for k in range(3)])
        rel = us - _solid_velocity(omega, center, x, y, z)
        utv = rel - rel.dot(N_HAT) * N_HAT
        utm = np.linalg.norm(utv)
        t_hat = utv / utm
        y1 = max(phi[z, y, x], 0.5)
        utau = _utau(utm, y1 + YS)
        uw = utau * _uplus(y1 * utau / NU)
        g = (utm - uw) / YS
        S_ref = 0.5 * g * (np.outer(t_hat, N_HAT) + np.outer(N_HAT, t_hat))
        assert abs(ut[bz, by, bx] / utau - 1) < 2e-5, (x, y, z, ut[bz, by, bx], utau)
        du = wm[0:3, bz, by, bx]
        assert np.abs(du - uw * t_hat).max() < 2e-5 * uw
        S6 = wm[3:9, bz, by, bx]
        S6_ref = np.array([S_ref[0, 0], S_ref[1, 1], S_ref[2, 2], S_ref[0, 1], S_ref[0, 2], S_ref[1, 2]])
        assert np.abs(S6 - S6_ref).max() < 2e-5 * abs(g)
        assert y1 * utau / NU > 55.0                  # the log region
        checked += 1
    assert checked > 40
    lat.close()
