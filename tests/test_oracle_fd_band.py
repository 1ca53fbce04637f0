"""Pins of the oracle's finite-difference strain across the porous band
(hybrid non-equilibrium with sigma < 1, Sec. 2.2: f^(1) is replaced, in the
share 1 - sigma, by the Chapman-Enskog term built from the rate of strain
S^FD = (grad u + grad u^T) / 2 of the resolved velocity).

* Central differences are exact on quadratic velocity fields: S^FD equals
  the analytic symmetric gradient at every interior cell (a dropped factor
  1/2, a one-cell step or a missing symmetrisation fails).
* At an open face the difference is one-sided, exact on linear fields.
* The discrete adjoint through the band (S^FD transposed onto the
  neighbours' populations) against finite differences of the forward.
* Consistency of the hybrid collision: for populations that are exactly
  f^eq + f^(1) of a linear shear (the Chapman-Enskog state, Pi^neq =
  -2 rho cs^2 tau S) at a band cell with u = u^B = 0, the local and the
  finite-difference non-equilibrium parts coincide, so the post-collision
  populations do not depend on sigma; with the shear of the populations
  doubled against the velocity field they do.
"""

import numpy as np
import pytest

import oracle as O
from workloads.rotor import BladeGrid

CS2 = 1.0 / 3.0


def _grid_fields(shape):
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return np.stack([x, y, z]).astype(np.float64)


def _quadratic(X, G, Hq, x0):
    """u_b = G_ba (x - x0)_a + Hq_bac (x - x0)_a (x - x0)_c; its gradient."""
    r = X - np.asarray(x0, dtype=np.float64).reshape(3, 1, 1, 1)
    u = np.einsum("ba,a...->b...", G, r) + np.einsum("bac,a...,c...->b...", Hq, r, r)
    grad = G[None, None, None] + np.einsum("bac,c...->...ab", Hq + Hq.transpose(0, 2, 1), r).transpose(0, 1, 2, 4, 3)
    return u, grad            # grad[..., b, a] = du_b / dx_a


@pytest.mark.parametrize("q", [19, 27])
def test_fd_strain_exact_on_quadratic_fields(q):
    rng = np.random.default_rng(5)
    shape = (14, 10, 12)
    o = O.Oracle(12, 10, 14, q=q, open_boundaries=False, u_in=0.0)
    X = _grid_fields(shape)
    G = rng.uniform(-4e-3, 4e-3, (3, 3))
    Hq = rng.uniform(-2e-4, 2e-4, (3, 3, 3))
    u, grad = _quadratic(X, G, Hq, (5.5, 4.5, 6.5))
    o.init_equilibrium(1.0, u)
    S = o.fd_strain()
    Sref = 0.5 * (grad + np.swapaxes(grad, -1, -2))
    inner = (slice(1, -1),) * 3          # away from the periodic wrap
    err = np.abs(S[inner] - Sref[inner]).max()
    assert err <= 1e-13, err
    assert np.abs(S - np.swapaxes(S, -1, -2)).max() == 0.0
    assert np.abs(Sref[inner]).max() > 1e-3


def test_fd_strain_one_sided_at_open_faces():
    rng = np.random.default_rng(6)
    shape = (12, 9, 10)
    o = O.Oracle(10, 9, 12, q=19, open_boundaries=True, flow_axis=2, u_in=0.0)
    X = _grid_fields(shape)
    G = rng.uniform(-4e-3, 4e-3, (3, 3))
    u, grad = _quadratic(X, G, np.zeros((3, 3, 3)), (4.0, 4.0, 5.0))
    o.init_equilibrium(1.0, u)
    S = o.fd_strain()
    Sref = 0.5 * (grad + np.swapaxes(grad, -1, -2))
    sl = (slice(None), slice(1, -1), slice(1, -1))      # all z incl. both open faces
    assert np.abs(S[sl] - Sref[sl]).max() <= 1e-13
    # the periodic wrap sees the jump of a non-periodic field: not exact there
    assert np.abs(S[:, 0, 1:-1] - Sref[:, 0, 1:-1]).max() > 1e-3


def _sphere():
    g = BladeGrid(sdf=np.full((2, 2, 2), 100.0, np.float32), origin=(0.0, 0.0, 0.0), spacing=0.5,
                  radius=1.0, hub_radius=0.0, chord_root=1.0, chord_tip=1.0)
    return O.make_rotor(g, center=(8.3, 8.1, 10.2), axis=2, omega=0.0, n_blades=0, hub_radius=4.0)


def _post_collision_at(q, sigma, shear_scale):
    """Post-collision populations of one band cell x_c after one step from the
    Chapman-Enskog state of u = G (x - x_c), read from the neighbours the
    populations streamed to."""
    nx, ny, nz, tau = 16, 16, 20, 0.6
    o = O.Oracle(nx, ny, nz, q=q, open_boundaries=False, u_in=0.0, tau_mo=tau, c_smag=0.0,
                 wall_model=False, sigma_band=sigma, rotors=[_sphere()])
    o.step(1)
    _, d, fl, _ = o.geometry()
    band = np.argwhere((fl & 1) != 0)
    zc, yc, xc = band[np.argmin(np.abs(d[tuple(band.T)] - 0.5))]
    assert 0.0 < d[zc, yc, xc] < 1.0
    X = _grid_fields((nz, ny, nx))
    G = np.array([[0.0, 2e-3, -1e-3], [1.5e-3, 0.0, 0.5e-3], [-0.5e-3, 1e-3, 0.0]])
    u, _ = _quadratic(X, G, np.zeros((3, 3, 3)), (xc, yc, zc))
    Ssym = 0.5 * (G + G.T)
    c, w, _ = O.lattice(q)
    f = np.empty((q, nz, ny, nx))
    for i in range(q):
        H2S = sum((c[i][a] * c[i][b] - CS2 * (a == b)) * Ssym[a, b] for a in range(3) for b in range(3))
        f[i] = w[i] * (1.0 + (np.einsum("a,a...->...", c[i], u)) / CS2
                       + (np.einsum("a,a...->...", c[i], u) ** 2) / (2 * CS2 ** 2)
                       - np.einsum("a...,a...->...", u, u) / (2 * CS2)) \
            - shear_scale * w[i] * tau / CS2 * H2S
    o.set_populations(f)
    o.step(1)
    ft = o.populations()
    return np.array([ft[i, (zc + c[i][2]) % nz, (yc + c[i][1]) % ny, (xc + c[i][0]) % nx] for i in range(q)])


@pytest.mark.parametrize("q", [19, 27])
def test_hybrid_band_collision_consistent_for_chapman_enskog_state(q):
    f1 = _post_collision_at(q, 1.0, 1.0)
    f0 = _post_collision_at(q, 0.0, 1.0)
    fh = _post_collision_at(q, 0.5, 1.0)
    assert np.abs(f0 - f1).max() <= 1e-15 * 50
    assert np.abs(fh - f1).max() <= 1e-15 * 50
    g1 = _post_collision_at(q, 1.0, 2.0)
    g0 = _post_collision_at(q, 0.0, 2.0)
    assert np.abs(g0 - g1).max() > 1e-5


def _sigma_objective(wl, T, navg, wT, wQ, wall_model, pitch=None, d0=None):
    o = O.from_workload(wl, sigma_band=0.5, wall_model=wall_model)
    if pitch is not None:
        o.freeze_sets(True)
        o.set_pitch(0, pitch)
    if d0 is not None:
        o.set_d0(d0)
    a = wl.flow_axis
    J = 0.0
    for s in range(T):
        o.step(1)
        if s >= T - navg:
            F, M, _, _ = o.forces()
            J += (wT * F[0, a] + wQ * M[0, a]) / navg
    return J


@pytest.mark.parametrize("wall_model", [False, True])
def test_adjoint_with_hybrid_band_matches_differences(wall_model):
    """Gradient with sigma = 0.5: the collision of a force cell off the wall
    set reads S^FD built from its axis neighbours' pre-collision velocities,
    so the adjoint hands part of its strain sensitivity to those neighbours.
    dJ/d(pitch) (frozen sets) and dJ/d(d0) at a band cell and at fluid
    neighbours of band cells against central differences of the FP64
    forward.  Dropping that transpose moves dJ/d(pitch) by 9 % and the
    neighbours' dJ/d(d0) by 0.4 to 35 % on this case."""
    from workloads.configs import Workload, _single
    wl = Workload("grad", 32, 32, 64, steps=16, rotors=_single(32, 32, 64, 10.0, 6.0))
    T, navg, wT, wQ = 8, 4, 1.0, 0.5
    o = O.from_workload(wl, sigma_band=0.5, wall_model=wall_model)
    J, gp, gd0 = o.adjoint(T, navg, [wT], [wQ])
    assert abs(J - _sigma_objective(wl, T, navg, wT, wQ, wall_model)) <= 1e-14 * max(1.0, abs(J))
    h = 1e-3
    fd = (_sigma_objective(wl, T, navg, wT, wQ, wall_model, pitch=h)
          - _sigma_objective(wl, T, navg, wT, wQ, wall_model, pitch=-h)) / (2 * h)
    assert abs(gp[0] - fd) < 5e-4 * abs(fd), (gp[0], fd)
    if wall_model:
        return
    ref = O.from_workload(wl, sigma_band=0.5, wall_model=False)
    ref.step(1)
    fl = ref.geometry()[2]
    band = np.argwhere((fl & 1) > 0)
    assert len(band) > 200
    picks = [tuple(band[len(band) // 3])]
    for b in band[::len(band) // 40]:
        for d in ((1, 0, 0), (0, 1, 0), (0, 0, 1), (-1, 0, 0), (0, -1, 0), (0, 0, -1)):
            c = tuple(int(b[k] + d[k]) for k in range(3))
            if fl[c] == 0:
                picks.append(c)
                break
        if len(picks) == 4:
            break
    assert len(picks) == 4
    hd = 1e-5
    for cell in picks:
        e = np.ones(ref.shape)
        e[cell] += hd
        Jp = _sigma_objective(wl, T, navg, wT, wQ, False, d0=e)
        e[cell] -= 2 * hd
        Jm = _sigma_objective(wl, T, navg, wT, wQ, False, d0=e)
        fdv = (Jp - Jm) / (2 * hd)
        assert abs(gd0[cell] - fdv) <= 1e-6 * abs(fdv) + 1e-9 * max(1.0, abs(J)), (cell, gd0[cell], fdv)
