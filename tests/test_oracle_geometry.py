"""Pins of the oracle's porosity embedding (Sec. 2.2.2 Definition "Lattice
Porosity", Sec. 3.1 reference grid; no GPU)."""

import math

import numpy as np
import pytest

import oracle as O
from workloads import BladeGrid, make_blade_grid


def test_porosity_definition(golden):
    eps = 2.0
    assert O.porosity(-5.0, eps) == 0.0
    assert O.porosity(-1.0, eps) == 0.0
    assert O.porosity(1.0, eps) == 1.0
    assert O.porosity(7.0, eps) == 1.0
    # the real wall is the level set d = 1/2 at phi = 0, for both transition functions
    assert O.porosity(0.0, eps) == golden["porosity_wall_level"]["value"]
    assert O.porosity(0.0, eps, linear=True) == 0.5
    phis = np.linspace(-0.999, 0.999, 41)
    lin = np.array([O.porosity(p, eps, linear=True) for p in phis])
    assert np.allclose(lin, phis / eps + 0.5)           # the printed s(phi)
    sm = np.array([O.porosity(p, eps) for p in phis])
    assert np.all(np.diff(sm) > 0)
    # smoothstep: continuous slope at both ends of the transition
    h = 1e-6
    for end in (-1.0, 1.0):
        slope = (O.porosity(end + h, eps) - O.porosity(end - h, eps)) / (2 * h)
        assert abs(slope) < 1e-5
    # odd symmetry about the wall: d(phi) + d(-phi) = 1
    assert np.allclose(sm + sm[::-1], 1.0)


def _linear_grid(alpha, beta, gamma, delta, spacing=0.5, n=(45, 41, 37), origin=(-11.0, -10.0, -9.0)):
    gx, gy, gz = n
    R = origin[0] + spacing * np.arange(gx)
    T = origin[1] + spacing * np.arange(gy)
    A = origin[2] + spacing * np.arange(gz)
    AA, TT, RR = np.meshgrid(A, T, R, indexing="ij")
    sdf = (alpha * RR + beta * TT + gamma * AA + delta).astype(np.float32)
    return BladeGrid(sdf=np.ascontiguousarray(sdf), origin=origin, spacing=spacing, radius=17.0,
                     hub_radius=0.0, chord_root=1.0, chord_tip=1.0)


def _blade_frame_point(x, center, axis, psi, pitch):
    """Rotor geometry stated as rotations: span e_R = cos(psi) e_b + sin(psi) e_c,
    tangent e_T = -sin(psi) e_b + cos(psi) e_c, axis e_A = e_a (b = a+1, c = a+2);
    pitch turns the section about e_R so the chord angle to the rotor plane grows."""
    a, b, c = axis, (axis + 1) % 3, (axis + 2) % 3
    r = np.asarray(x, float) - np.asarray(center, float)
    eR = np.zeros(3); eR[b], eR[c] = math.cos(psi), math.sin(psi)
    eT = np.zeros(3); eT[b], eT[c] = -math.sin(psi), math.cos(psi)
    eA = np.zeros(3); eA[a] = 1.0
    p = np.array([r @ eR, r @ eT, r @ eA])
    P = np.array([[1, 0, 0],
                  [0, math.cos(pitch), -math.sin(pitch)],
                  [0, math.sin(pitch), math.cos(pitch)]])
    return P @ p, (eR, eT, eA, P)


@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("pitch", [0.0, 0.13, -0.4])
def test_embedding_of_linear_field(axis, pitch):
    """Trilinear sampling reproduces a linear field exactly, so the embedded
    value at every cell is the linear function of its blade-frame position
    (azimuth theta0 + Omega t, then pitch)."""
    coef = (0.3, -0.7, 0.5, 0.25)
    g = _linear_grid(*coef)
    center = [20.5, 19.0, 21.5]
    omega, phase0, t = 0.031, 0.4, 17
    rot = O.make_rotor(g, center=center, axis=axis, omega=omega, phase0=phase0, pitch=pitch,
                       n_blades=1, hub_radius=0.0)
    rng = np.random.default_rng(7)
    xyz = rng.integers(10, 32, size=(300, 3))
    phi, which = O.rotor_phi(rot, t, xyz)
    psi = phase0 + omega * t
    n_checked = 0
    for k in range(len(xyz)):
        q, _ = _blade_frame_point(xyz[k], center, axis, psi, pitch)
        lo = np.array(g.origin)
        hi = lo + g.spacing * (np.array(g.sdf.shape[::-1]) - 1)
        if np.any(q < lo - 1e-3) or np.any(q > hi + 1e-3):
            assert phi[k] == np.inf          # outside the reference grid: no solid
            continue
        if np.any(q < lo + 1e-3) or np.any(q > hi - 1e-3):
            continue                         # on the grid boundary: either side is valid
        want = coef[0] * q[0] + coef[1] * q[1] + coef[2] * q[2] + coef[3]
        assert abs(phi[k] - want) < 2e-5 * (1 + abs(want))
        assert which[k] == 0
        n_checked += 1
    assert n_checked > 100
    # outward normal: the rotated gradient direction of the linear field
    x = xyz[0]
    _, (eR, eT, eA, P) = _blade_frame_point(x, center, axis, psi, pitch)
    gq = np.array(coef[:3])
    gp = P.T @ gq
    glab = gp[0] * eR + gp[1] * eT + gp[2] * eA
    n = O.rotor_normal(rot, t, 0, *x)
    assert np.allclose(n, glab / np.linalg.norm(glab), atol=1e-12)


def test_hub_sphere_distance_and_normal():
    g = _linear_grid(0, 0, 0, 100.0)
    center = [15.5, 16.0, 14.25]
    rot = O.make_rotor(g, center=center, axis=2, omega=0.05, n_blades=0, hub_radius=6.0)
    xs = np.stack(np.meshgrid(np.arange(32), np.arange(32), np.arange(32), indexing="ij"), -1).reshape(-1, 3)
    for t in (0, 9, 123):
        phi, which = O.rotor_phi(rot, t, xs)
        want = np.linalg.norm(xs - np.array(center), axis=1) - 6.0
        assert np.abs(phi - want).max() < 1e-5
        assert np.all(which == 0)          # index n_blades = hub
    n = O.rotor_normal(rot, 0, 0, 3, 4, 5)
    r = np.array([3, 4, 5]) - np.array(center)
    assert np.allclose(n, r / np.linalg.norm(r), atol=1e-14)


def test_threefold_symmetry_and_sense_of_rotation():
    """The three-bladed rotor looks the same after a third of a turn, and its
    blades move in the sense of the solid velocity Omega a x (x - c)."""
    g = make_blade_grid(12.0)
    center = (23.5, 23.5, 24.0)
    omega = 0.025

    def mk(ph):
        return O.make_rotor(g, center=center, axis=2, omega=omega, phase0=ph)

    xs = np.stack(np.meshgrid(np.arange(4, 44), np.arange(4, 44), np.arange(14, 35), indexing="ij"),
                  -1).reshape(-1, 3)
    p0, _ = O.rotor_phi(mk(0.3), 5, xs)
    p1, _ = O.rotor_phi(mk(0.3 + 2 * math.pi / 3), 5, xs)
    fin = np.isfinite(p0)
    assert np.abs(p0[fin] - p1[fin]).max() < 1e-4
    # sense of rotation: mean azimuth of blade 0's transition cells advances by +Omega dt
    rot = mk(0.0)

    def azimuth(t):
        p, w = O.rotor_phi(rot, t, xs)
        sel = (p < 1.0) & (w == 0)
        r = xs[sel] - np.array(center)
        rr = np.hypot(r[:, 0], r[:, 1])
        sel2 = rr > 6
        return math.atan2(np.sum(r[sel2, 1] / rr[sel2]), np.sum(r[sel2, 0] / rr[sel2]))

    dt = 24
    dpsi = azimuth(dt) - azimuth(0)
    assert abs(dpsi - omega * dt) < 0.15 * omega * dt
