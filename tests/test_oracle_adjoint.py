"""Pins of the oracle's discrete adjoint (no GPU).

The adjoint's local Jacobians are taken by complex-step differentiation, so
they are checked here against things computed without it: real central
differences of the FP64 forward, the conservation laws of the collision
(which fix the adjoint of mass and momentum in closed form), and central
differences of the whole objective J with the cell sets held fixed (the
reading for the set memberships, which otherwise make J jump).  The pitch
enters the forward through a binary32 signed distance, so pitch differences
use h = 1e-3 rad; the static multiplier d0 enters in FP64 and takes
h = 1e-6.
"""

import numpy as np
import pytest

import oracle as O
import workloads as W
from workloads import random_populations
from workloads.configs import RotorSpec, Workload, _single


def _cells(q, n, seed):
    c, w, _ = O.lattice(q)
    rng = np.random.default_rng(seed)
    u = rng.normal(0.0, 0.05, (n, 3))
    f = np.stack([O.equilibrium(q, 1.0 + 0.02 * rng.uniform(-1, 1), u[k]) for k in range(n)])
    return f + random_populations(seed, n, w, 2e-3), rng


@pytest.mark.parametrize("q", [19, 27])
def test_collide_vjp_matches_central_differences(q):
    """Complex-step VJP of the hybrid collision (Eq. (hlbm)) against real
    central differences of the FP64 forward, for bulk, band (sigma = 1 and
    0.9) and wall (sigma = 0 with S^FD) cells."""
    n = 4
    f, rng = _cells(q, n, 3)
    d = np.array([1.0, 0.7, 0.3, 0.5])
    uB = rng.normal(0, 0.03, (n, 3))
    sig = np.array([1.0, 1.0, 0.9, 0.0])
    S = rng.normal(0, 1e-3, (n, 3, 3))
    lam = rng.normal(0, 1, (n, q))
    lf, gd, gu, gS = O.collide_vjp_cells(q, f, lam, d, uB, sig, S)
    h = 1e-6

    def L(ff=f, dd=d, uu=uB, SS=S):
        out, _ = O.collide_cells(q, ff, dd, uu, sig, SS)
        return (out * lam).sum(1)

    for j in range(q):
        e = np.zeros_like(f)
        e[:, j] = h
        np.testing.assert_allclose(lf[:, j], (L(ff=f + e) - L(ff=f - e)) / (2 * h), rtol=0, atol=2e-8)
    np.testing.assert_allclose(gd, (L(dd=d + h) - L(dd=d - h)) / (2 * h), rtol=0, atol=2e-9)
    for k in range(3):
        e = np.zeros_like(uB)
        e[:, k] = h
        np.testing.assert_allclose(gu[:, k], (L(uu=uB + e) - L(uu=uB - e)) / (2 * h), rtol=0, atol=2e-9)
    for a in range(3):
        for b in range(3):
            e = np.zeros_like(S)
            e[:, a, b] = h
            np.testing.assert_allclose(gS[:, a, b], (L(SS=S + e) - L(SS=S - e)) / (2 * h), rtol=0, atol=2e-9)


@pytest.mark.parametrize("q", [19, 27])
def test_collide_vjp_conservation(q):
    """The collision keeps the mass, sum f* = rho, and sets the momentum to
    sum c f* = rho u^ with u^ = d u + (1 - d) u^B (Eq. (convexVelocity)).
    So for lam* = 1 the adjoint is lam = 1 with no parameter sensitivity, and
    for lam* = c_a it is lam_i = d c_ia + (1 - d) u^B_a, g_d = rho (u - u^B)_a,
    g_uB = rho (1 - d) e_a, g_S = 0."""
    c, w, _ = O.lattice(q)
    n = 4
    f, rng = _cells(q, n, 5)
    d = np.array([1.0, 0.6, 0.2, 0.9])
    uB = rng.normal(0, 0.03, (n, 3))
    sig = np.array([1.0, 0.9, 0.0, 1.0])
    S = rng.normal(0, 1e-3, (n, 3, 3))
    lf, gd, gu, gS = O.collide_vjp_cells(q, f, np.ones((n, q)), d, uB, sig, S)
    np.testing.assert_allclose(lf, 1.0, atol=1e-12)
    assert np.abs(gd).max() < 1e-12 and np.abs(gu).max() < 1e-12 and np.abs(gS).max() < 1e-12
    rho = f.sum(1)
    u = f @ c / rho[:, None]
    for a in range(3):
        lf, gd, gu, gS = O.collide_vjp_cells(q, f, np.broadcast_to(c[:, a], (n, q)), d, uB, sig, S)
        want = d[:, None] * c[None, :, a] + ((1 - d) * uB[:, a])[:, None]
        np.testing.assert_allclose(lf, want, atol=1e-12)
        np.testing.assert_allclose(gd, rho * (u[:, a] - uB[:, a]), atol=1e-12)
        e = np.zeros(3)
        e[a] = 1.0
        np.testing.assert_allclose(gu, (rho * (1 - d))[:, None] * e, atol=1e-12)
        assert np.abs(gS).max() < 1e-12


def _wl(nz=64):
    return Workload("grad", 32, 32, nz, steps=16, rotors=_single(32, 32, nz, 10.0, 6.0))


def _objective(wl, T, navg, wT, wQ, pitch=None, d0=None, wall_model=True):
    o = O.from_workload(wl, wall_model=wall_model)
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


def test_porosity_and_normal_tangents_match_forward():
    """d(d)/d(pitch) of every force-set cell and dn/d(pitch) of wall cells
    (complex step, Sec. 3.1 geometry) against central differences of the
    forward with frozen sets."""
    wl = _wl()
    h = 1e-3

    def geo(p):
        o = O.from_workload(wl)
        o.freeze_sets(True)
        o.set_pitch(0, p)
        o.step(1)
        return o

    o0 = geo(0.0)
    _, d0, fl, _ = o0.geometry()
    tan = o0.porosity_tangent()
    fd = (geo(h).geometry()[1] - geo(-h).geometry()[1]) / (2 * h)
    B = (fl & 1) > 0
    assert B.sum() > 100
    scale = np.abs(tan[B]).max()
    assert np.abs(fd - tan)[B].max() < 1e-3 * scale
    assert np.abs(tan[~B]).max() == 0.0
    grid = wl.blade_grids()[0]
    spec = wl.rotors[0]
    worst = 0.0
    for (x, y, z, which) in [(8, 16, 10, 0), (23, 14, 16, 1), (16, 20, 15, 2), (17, 12, 9, 0)]:
        def nrm(p):
            r = O.make_rotor(grid, center=spec.center, axis=2, omega=spec.omega(wl.u_in), pitch=p)
            return O.rotor_normal(r, 0, which, x, y, z)
        r0 = O.make_rotor(grid, center=spec.center, axis=2, omega=spec.omega(wl.u_in), pitch=0.0)
        dn = O.rotor_normal_tangent(r0, 0, which, x, y, z)
        fdn = (nrm(1e-5) - nrm(-1e-5)) / 2e-5
        worst = max(worst, np.abs(dn - fdn).max() / max(1e-3, np.abs(fdn).max()))
    assert worst < 1e-5


def test_wall_model_tangent_matches_forward():
    """d du_WM/d(pitch) and d S_WM/d(pitch) of every active wall cell of the
    first step (cold Newton starts, some of them stopped by the iteration
    cap at blade speed), complex step through the two Newton solves as
    iterated, against central differences of the forward."""
    wl = _wl()
    h = 1e-3

    def fresh(p):
        o = O.from_workload(wl)
        o.freeze_sets(True)
        o.set_pitch(0, p)
        return o

    ddu, dS = fresh(0.0).wall_tangent()
    plus, minus = fresh(h), fresh(-h)
    plus.step(1)
    minus.step(1)
    a, b = plus.wall_state(), minus.wall_state()
    ref = fresh(0.0)
    ref.step(1)
    act = ref.wall_state()[3] > 0
    assert act.sum() > 100
    fdu = (a[0] - b[0]) / (2 * h)
    fS = (a[1] - b[1]) / (2 * h)
    # relative L2 over the wall cells (the trilinear blade grid has kinks
    # that a few cells cross within +-h)
    assert np.linalg.norm((fdu - ddu)[act]) < 1e-2 * np.linalg.norm(ddu[act])
    assert np.linalg.norm((fS - dS)[act]) < 1e-2 * np.linalg.norm(dS[act])


def test_adjoint_pitch_matches_frozen_differences():
    """dJ/d(pitch) of J = mean over the last 4 of 8 steps of thrust + 0.5 torque,
    wall model on, against central differences (h = 1e-3 rad) of the forward
    with the cell sets frozen."""
    wl = _wl()
    T, navg, wT, wQ = 8, 4, 1.0, 0.5
    o = O.from_workload(wl)
    J, gp, _ = o.adjoint(T, navg, [wT], [wQ])
    assert abs(J - _objective(wl, T, navg, wT, wQ)) <= 1e-14 * max(1.0, abs(J))
    h = 1e-3
    fd = (_objective(wl, T, navg, wT, wQ, pitch=h) - _objective(wl, T, navg, wT, wQ, pitch=-h)) / (2 * h)
    assert abs(gp[0] - fd) < 5e-4 * abs(fd), (gp[0], fd)
    # the state ends where the forward ends
    ref = O.from_workload(wl)
    ref.step(T)
    assert np.array_equal(o.populations(), ref.populations())


def test_adjoint_d0_matches_differences():
    """dJ/d(d0) at bulk, band, wall and wall-model-sample cells and at the
    outlet's upstream plane, for a rotor close to the outlet (the outlet
    equilibrium takes that plane's velocity of the previous step, a route
    worth a few per cent of those cells' gradient here), against FP64
    central differences (h = 1e-5)."""
    wl = Workload("grad_outlet", 32, 32, 28, steps=12,
                  rotors=[RotorSpec(center=(15.5, 15.5, 19.0), radius=10.0, tsr=6.0)])
    T, navg, wT, wQ = 12, 6, 1.0, -0.3
    o = O.from_workload(wl)
    J, gp, gd0 = o.adjoint(T, navg, [wT], [wQ])
    ref = O.from_workload(wl)
    ref.step(1)
    _, dfield, fl, _ = ref.geometry()
    band = np.argwhere((fl & 1) > 0)
    wall = np.argwhere((fl & 2) > 0)
    picks = [tuple(band[len(band) // 3]), tuple(band[2 * len(band) // 3]), tuple(wall[len(wall) // 2])]
    picks += [(12, 16, 16), (19, 3, 16), (26, 16, 16), (26, 20, 12), (25, 16, 16)]
    h = 1e-5
    for cell in picks:
        e = np.ones(ref.shape)
        e[cell] += h
        Jp = _objective(wl, T, navg, wT, wQ, d0=e)
        e[cell] -= 2 * h
        Jm = _objective(wl, T, navg, wT, wQ, d0=e)
        fd = (Jp - Jm) / (2 * h)
        # central-difference rounding: a few ulps of J over 2h
        assert abs(gd0[cell] - fd) <= 1e-6 * abs(fd) + 1e-9 * max(1.0, abs(J)), (cell, gd0[cell], fd)
        assert abs(fd) > 1e-5, cell
