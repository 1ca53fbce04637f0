"""Pins of the oracle's torque-driven rotor ("evolve structure" of the
listing "HHRRLBM-FSI" as rigid rotation, I dOmega/dt = M.a - Q_gen).

A sphere spun in a periodic box of fluid at rest is slowed by the viscous
torque.  Its magnitude is pinned against the Stokes rotlet torque
8 pi mu a^3 Omega (larger in a periodic box: the images and the finite box
add drag); the spin-down of the driven sphere is pinned against the decay
that the torque measured under prescribed rotation predicts (the flow is
quasi-steady: the decay time is 20 times the viscous time a^2 / nu); the
generator torque enters with its sign.  In the limit of infinite inertia the
driven rotor is the prescribed rotor.
"""

import numpy as np

import oracle as O
import workloads as W
from workloads.configs import Workload, _single
from workloads.rotor import BladeGrid


def _no_blades():
    return BladeGrid(sdf=np.full((2, 2, 2), 100.0, np.float32), origin=(0.0, 0.0, 0.0), spacing=0.5,
                     radius=1.0, hub_radius=0.0, chord_root=1.0, chord_tip=1.0)


def test_infinite_inertia_is_prescribed_rotation():
    wl = Workload("drive", 32, 32, 64, steps=12, rotors=_single(32, 32, 64, 10.0, 6.0))
    a = O.from_workload(wl)
    b = O.from_workload(wl)
    b.set_drive(0, 1e300)
    a.step(12)
    b.step(12)
    om = wl.rotors[0].omega(wl.u_in)
    th, omb = b.drive_state(0)
    assert omb == om
    assert abs(th - 12 * om) <= 1e-15
    fa, fb = a.populations(), b.populations()
    assert np.abs(fa - fb).max() <= 1e-13


def _spinning_sphere(om0=0.004, a=5.0, tau=0.8):
    rot = O.make_rotor(_no_blades(), center=(15.5, 15.5, 15.5), axis=2, omega=om0, n_blades=0, hub_radius=a)
    o = O.Oracle(32, 32, 32, open_boundaries=False, tau_mo=tau, c_smag=0.0, u_in=0.0, wall_model=False,
                 rotors=[rot])
    o.step(400)                      # prescribed rotation: the flow settles (a^2 / nu = 250 steps)
    _, M, _, _ = o.forces()
    return o, M[0, 2]


def test_sphere_torque_and_spin_down():
    om0, a, tau = 0.004, 5.0, 0.8
    nu = (tau - 0.5) / 3.0
    o, T0 = _spinning_sphere(om0, a, tau)
    stokes = -8.0 * np.pi * nu * a ** 3 * om0
    assert 1.0 <= T0 / stokes <= 1.25, T0 / stokes
    lam = 3e-4                       # decay rate the prescribed torque implies for this inertia
    inertia = -T0 / (lam * om0)
    o.set_drive(0, inertia)
    o.step(300)
    th, om = o.drive_state(0)
    assert abs(om / om0 - np.exp(-lam * 300)) <= 3e-3 * np.exp(-lam * 300)
    assert th > 0.0


def test_generator_torque_sign_and_magnitude():
    """Q_gen = k Omega |Omega| adds to the viscous torque: the driven sphere
    follows the explicit Euler solution of I dOmega/dt = c Omega - k Omega^2
    with the quasi-steady viscous coefficient c = T0 / Omega0."""
    om0 = 0.004
    o, T0 = _spinning_sphere(om0)
    c = T0 / om0
    inertia = -T0 / (3e-4 * om0)
    k_gen = -c / om0                 # generator torque equal to the viscous torque at Omega0
    o.set_drive(0, inertia, k_gen=k_gen)
    o.step(300)
    _, om = o.drive_state(0)
    ref = om0
    for _ in range(300):
        ref = ref + (c * ref - k_gen * ref * abs(ref)) / inertia
    assert abs(om - ref) <= 5e-3 * ref, (om, ref)
    assert om < om0 * np.exp(-3e-4 * 300)      # slower than without the generator
