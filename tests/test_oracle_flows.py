"""Whole-lattice pins of the oracle (no GPU): analytic flows, invariants and
balances that the scheme must satisfy independently of how it is coded."""

import math

import numpy as np
import pytest

import oracle as O
from workloads import BladeGrid, fourier_modes, make_blade_grid


def _dummy_grid():
    return BladeGrid(sdf=np.full((2, 2, 2), 100.0, np.float32), origin=(0.0, 0.0, 0.0), spacing=0.5,
                     radius=1.0, hub_radius=0.0, chord_root=1.0, chord_tip=1.0)


def _slab_grid(n, c, a, b, h=0.5):
    """Static geometry through the rotor machinery (Omega = 0, theta = 0,
    axis z): blade frame (R, T, A) = lab (x, y, z) - c.  Solid for y < a and
    y > b: phi = min(y - a, b - y)."""
    lo = [-c[k] - 2 for k in range(3)]
    hi = [n[k] - 1 - c[k] + 2 for k in range(3)]
    g = [int(round((hi[k] - lo[k]) / h)) + 1 for k in range(3)]
    R = lo[0] + h * np.arange(g[0])
    T = lo[1] + h * np.arange(g[1])
    A = lo[2] + h * np.arange(g[2])
    AA, TT, RR = np.meshgrid(A, T, R, indexing="ij")
    y = TT + c[1]
    sdf = np.minimum(y - a, b - y).astype(np.float32)
    return BladeGrid(sdf=np.ascontiguousarray(sdf), origin=tuple(lo), spacing=h, radius=1.0,
                     hub_radius=0.0, chord_root=1.0, chord_tip=1.0)


def _cylinder_grid(half, nz, cz, sign, radius, h=0.5):
    """Axis-z cylinder as a blade-frame level set (one 'blade', no hub):
    sign = +1 is solid inside r < radius, sign = -1 solid outside r > radius;
    the grid spans +-half across the axis and the whole periodic length."""
    lo = [-half, -half, -cz - 2]
    hi = [half, half, nz - 1 - cz + 2]
    g = [int(round((hi[k] - lo[k]) / h)) + 1 for k in range(3)]
    R = lo[0] + h * np.arange(g[0])
    T = lo[1] + h * np.arange(g[1])
    A = lo[2] + h * np.arange(g[2])
    _, TT, RR = np.meshgrid(A, T, R, indexing="ij")
    sdf = (sign * (np.hypot(RR, TT) - radius)).astype(np.float32)
    return BladeGrid(sdf=np.ascontiguousarray(sdf), origin=tuple(lo), spacing=h, radius=1.0,
                     hub_radius=0.0, chord_root=1.0, chord_tip=1.0)


def _tgv_viscosity_error(n, tau=0.8, U0=0.01):
    o = O.Oracle(n, n, 2, open_boundaries=False, tau_mo=tau, c_smag=0.0, u_in=0.0, wall_model=False)
    k = 2 * math.pi / n
    x = np.arange(n)
    Z, Y, X = np.meshgrid(np.arange(2), x, x, indexing="ij")
    ux = -U0 * np.cos(k * X) * np.sin(k * Y)
    uy = U0 * np.sin(k * X) * np.cos(k * Y)
    rho = 1 - 3 * U0**2 / 4 * (np.cos(2 * k * X) + np.cos(2 * k * Y))
    o.init_equilibrium(rho, np.stack([ux, uy, 0 * ux]))

    def energy():
        r, u = o.fields()
        return 0.5 * np.sum(r * (u**2).sum(0))

    t1, t2 = 100, int(1000 * (n / 64) ** 2)
    o.step(t1)
    e1 = energy()
    o.step(t2 - t1)
    e2 = energy()
    nu = (tau - 0.5) / 3
    return math.log(e1 / e2) / (4 * k * k * (t2 - t1)) / nu - 1


def test_taylor_green_viscosity_second_order():
    """2D Taylor-Green vortex on a periodic box (C_S = 0, d = 1): kinetic
    energy decays as exp(-4 nu k^2 t) with the lattice viscosity
    nu = (tau - 1/2)/3, and the error falls with the square of the spacing."""
    e32 = _tgv_viscosity_error(32)
    e64 = _tgv_viscosity_error(64)
    assert abs(e64) < 1e-3
    assert abs(e32) / abs(e64) > 3.0


def test_rest_state_and_uniform_flow_are_fixed_points():
    o = O.Oracle(6, 5, 7, open_boundaries=False, u_in=0.0, wall_model=False)
    o.init_equilibrium(1.0, np.zeros(3)[:, None, None, None])
    c, w, _ = O.lattice(19)
    o.step(200)
    assert np.abs(o.populations() - w[:, None, None, None]).max() < 1e-15
    u0 = np.array([0.03, -0.02, 0.05])
    o = O.Oracle(6, 5, 7, open_boundaries=False, wall_model=False)
    o.init_equilibrium(1.0, u0[:, None, None, None])
    o.step(200)
    rho, u = o.fields()
    assert np.abs(rho - 1).max() < 1e-14
    assert np.abs(u - u0[:, None, None, None]).max() < 1e-14


def _periodic_rotor(wall_model=False, omega=0.025):
    g = make_blade_grid(12.0)
    rot = O.make_rotor(g, center=(23.5, 23.5, 24.0), axis=2, omega=omega)
    return O.Oracle(48, 48, 48, open_boundaries=False, wall_model=wall_model, rotors=[rot])


def test_mass_conservation_with_rotating_rotor():
    """Collision conserves mass in every cell and streaming permutes
    populations, so on a periodic box the total mass is constant to roundoff
    with porosity, rotation and the wall model active."""
    o = _periodic_rotor(wall_model=True)
    m0 = o.mass()
    o.step(30)
    assert abs(o.mass() - m0) / m0 < 1e-13


def test_momentum_balance_per_step():
    """On a periodic box the total fluid momentum changes in one step by the
    homogenized forcing only: sum_x rho (1 - d) (u^B - u), u^B = Omega a x (x - c).
    Sums are taken exactly rounded (math.fsum) so that only the oracle's
    per-cell rounding remains."""
    o = _periodic_rotor(wall_model=False)
    o.step(10)
    Z, Y, X = np.meshgrid(np.arange(48), np.arange(48), np.arange(48), indexing="ij")
    us = np.stack([-0.025 * (Y - 23.5), 0.025 * (X - 23.5), 0 * X])

    def total(a):
        return np.array([math.fsum(a[k].ravel()) for k in range(3)])

    for _ in range(3):
        rho, u = o.fields()
        P0 = total(rho * u)
        o.step(1)
        _, d, fl, _ = o.geometry()
        rho1, u1 = o.fields()
        P1 = total(rho1 * u1)
        forcing = total(rho * (1 - d) * (us - u))
        scale = total(rho * (1 - d) * np.abs(us - u)).max()
        assert np.abs((P1 - P0) - forcing).max() < 1e-11 * scale
        assert np.all((d < 1) == ((fl & 1) == 1))


@pytest.mark.parametrize("form", [0, 1])
def test_momentum_exchange_matches_deficit_at_steady_state(form):
    """A fixed sphere in a channel at steady state: the Galilean-invariant link
    form of the momentum exchange (the reading of Sec. 2.2.2) equals the
    momentum the homogenized forcing removes, sum rho (1 - d) u; the printed
    sign pattern taken literally does not."""
    rot = O.make_rotor(_dummy_grid(), center=(11.5, 11.5, 14.0), axis=2, omega=0.0, n_blades=0,
                       hub_radius=3.0)
    o = O.Oracle(24, 24, 48, tau_mo=0.6, c_smag=0.0, u_in=0.05, wall_model=False, rotors=[rot],
                 force_form=form)
    o.step(800)
    rho, u = o.fields()
    o.step(1)
    F, M, _, _ = o.forces()
    _, d, _, _ = o.geometry()
    D = np.array([np.sum(rho * (1 - d) * u[k]) for k in range(3)])
    assert D[2] > 0                                      # drag points downstream
    if form == 0:
        assert abs(F[0, 2] - D[2]) < 1e-3 * D[2]
        assert np.abs(F[0, :2]).max() < 1e-10 * D[2]     # symmetric body: no side force
    else:
        assert abs(F[0, 2] - D[2]) > 0.5 * D[2]


def test_rotating_sphere_symmetry_and_torque_sign():
    """A sphere spun in fluid at rest: no net force by symmetry and a torque
    that opposes the rotation (the fluid is dragged along)."""
    rot = O.make_rotor(_dummy_grid(), center=(15.5, 15.5, 15.5), axis=2, omega=0.01, n_blades=0,
                       hub_radius=5.0)
    o = O.Oracle(32, 32, 32, open_boundaries=False, tau_mo=0.55, c_smag=0.1, u_in=0.0,
                 wall_model=False, rotors=[rot])
    o.step(40)
    F, M, _, _ = o.forces()
    assert M[0, 2] < 0
    assert np.abs(F[0]).max() < 1e-5 * abs(M[0, 2]) / 5.0
    assert np.abs(M[0, :2]).max() < 1e-4 * abs(M[0, 2])


def test_circular_couette_profile_and_torque():
    """Laminar flow between a porous cylinder of radius R1 spun at Omega (its
    cells move with u^B = Omega a x (x - c), Sec. 2.2) and a fixed porous
    outer wall at R2, periodic along the axis.  Steady state: the Navier-Stokes
    solution u_theta = A r + B / r with u_theta(R1) = Omega R1, u_theta(R2) = 0
    (walls at the d = 1/2 level sets), no radial flow, and a torque per unit
    length 4 pi mu Omega R1^2 R2^2 / (R2^2 - R1^2) on each wall, opposite in
    sign: the fluid resists the inner cylinder and drags the outer one.  The
    diffuse interface (2 cells) and the staircase of a 12-cell gap leave a
    few per cent; a wrong sign of u^B, a dropped (1 - d) u^B or a wrong lever
    arm in the torque sum each fails by far more."""
    n, nz, c = 48, 2, (23.5, 23.5, 0.5)
    R1, R2, Om, tau = 8.0, 20.0, 0.0025, 0.8
    inner = O.make_rotor(_cylinder_grid(R1 + 4, nz, c[2], 1, R1), center=c, axis=2, omega=Om, n_blades=1,
                         hub_radius=0.0)
    outer = O.make_rotor(_cylinder_grid(36.0, nz, c[2], -1, R2), center=c, axis=2, omega=0.0, n_blades=1,
                         hub_radius=0.0)
    o = O.Oracle(n, n, nz, open_boundaries=False, tau_mo=tau, c_smag=0.0, u_in=0.0, wall_model=False,
                 rotors=[inner, outer])
    o.step(1500)      # about ten e-folding times gap^2 / (pi^2 nu) of the spin-up
    _, u = o.fields()
    Y, X = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    dx, dy = X - c[0], Y - c[1]
    r = np.hypot(dx, dy)
    ut = (-dy * u[0, 0] + dx * u[1, 0]) / r
    ur = (dx * u[0, 0] + dy * u[1, 0]) / r
    A = -Om * R1**2 / (R2**2 - R1**2)
    B = Om * R1**2 * R2**2 / (R2**2 - R1**2)
    sel = (r >= R1 + 1) & (r <= R2 - 1)
    assert np.abs(ut[sel] - (A * r[sel] + B / r[sel])).max() < 0.05 * Om * R1
    assert np.abs(ur[sel]).max() < 0.01 * Om * R1
    assert np.array_equal(u[:, 0], u[:, 1])                       # uniform along the axis
    F, M, _, _ = o.forces()
    nu = (tau - 0.5) / 3.0
    Tq = 4.0 * math.pi * nu * Om * R1**2 * R2**2 / (R2**2 - R1**2) * nz
    assert 0.97 < -M[0, 2] / Tq < 1.08
    assert abs(M[0, 2] + M[1, 2]) < 1e-3 * Tq                   # steady: the fluid passes the torque on
    assert np.abs(F).max() < 1e-6 * Tq / R1                       # no net force by symmetry
    assert np.abs(M[:, :2]).max() < 1e-6 * Tq


@pytest.mark.parametrize("wall_model", [False, True])
def test_porous_channel_profile(wall_model):
    """Uniform inflow into a channel between two porous slabs develops the
    plane Poiseuille profile; its zero crossings sit at the d = 1/2 level sets
    (the real wall, Definition "Lattice Porosity") to a fraction of a cell,
    with the wall model off and on (laminar flow sits in the sublayer)."""
    n = (2, 24, 64)
    c = (0.5, 11.5, 32.0)
    a, b = 3.5, 19.5
    rot = O.make_rotor(_slab_grid(n, c, a, b), center=c, axis=2, omega=0.0, n_blades=1, hub_radius=0.0)
    o = O.Oracle(*n, tau_mo=0.8, c_smag=0.0, u_in=0.02, wall_model=wall_model, rotors=[rot])
    o.step(3000)
    _, u = o.fields()
    prof = u[2, 44, :, 0]
    prof2 = u[2, 52, :, 0]
    ys = np.arange(n[1])
    sel = (ys >= a + 1.5) & (ys <= b - 1.5)
    p = np.polyfit(ys[sel], prof[sel], 2)
    roots = np.sort(np.roots(p).real)
    assert np.abs(np.polyval(p, ys[sel]) - prof[sel]).max() < 2e-3 * prof.max()
    assert abs(roots[0] - a) < 0.3 and abs(roots[1] - b) < 0.3
    assert np.abs(prof - prof2).max() < 1e-2 * prof.max()      # developed
    assert np.abs(u[2, 44, :2, 0]).max() < 1e-2 * prof.max()   # at rest inside the solid


def test_turbulent_inflow_statistics():
    """Synthetic inflow: the mode table is divergence-free (k . a = k . b = 0)
    and the evaluated inlet velocity has mean U along the axis and a
    per-component rms near the requested 5 % of U."""
    U = 0.05
    modes = fourier_modes(3, 64, 128.0, U, 0.05)
    assert np.abs(np.sum(modes[:, 0:3] * modes[:, 3:6], 1)).max() < 1e-15
    assert np.abs(np.sum(modes[:, 0:3] * modes[:, 6:9], 1)).max() < 1e-15
    o = O.Oracle(64, 64, 4, u_in=U, modes=modes, wall_model=False)
    samples = np.stack([o.inflow_plane(t) for t in range(0, 4000, 97)])
    mean = samples.reshape(-1, 3).mean(0)
    assert abs(mean[2] - U) < 0.1 * 0.05 * U
    rms = samples.reshape(-1, 3).std(0)
    assert np.all(np.abs(rms / (0.05 * U) - 1) < 0.35)
    assert abs(rms.mean() / (0.05 * U) - 1) < 0.2


def test_inflow_plane_input_matches_oracle():
    """The host evaluation of the synthetic inflow (input data for a caller's
    inflow plane) equals the oracle's inlet velocities, flow along z and x."""
    from workloads.turbulence import fourier_modes, inflow_plane
    for shape, axis in (((12, 10, 20), 2), ((20, 12, 10), 0)):
        modes = fourier_modes(3, 16, float(shape[axis]), 0.05, 0.05)
        o = O.Oracle(*shape, flow_axis=axis, u_in=0.05, modes=modes)
        for t in (0, 7, 31):
            ref = o.inflow_plane(t)                     # (n_c, n_b, 3)
            got = inflow_plane(modes, shape, axis, 0.05, t)
            assert np.abs(got.transpose(1, 2, 0) - ref).max() <= 1e-15
            assert np.abs(got - 0.05 * (np.arange(3) == axis)[:, None, None]).max() > 1e-4
