"""Torque-driven rotors on the GPU (evolve structure on the device) against
the FP64 oracle: angular velocity and angle trajectories, fields, the
infinite-inertia limit, spin-down of a sphere, snapshots, and the gradient
call's refusal."""

import numpy as np
import pytest

import oracle as O
import workloads as W
from workloads.rotor import BladeGrid

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("a CUDA device is required for the gpu-marked tests")
    from paper_2510_13726_b300.build import build
    build()
    import paper_2510_13726_b300 as pkg
    return pkg


def _rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def test_driven_rotor_matches_oracle(P):
    """rotor48 (R = 12, TSR 6) turning under its own torque and a generator
    law for 60 steps; the inertia makes Omega change by several per cent."""
    wl = W.workload("rotor48")
    om0 = wl.rotors[0].omega(wl.u_in)
    probe = O.from_workload(wl)
    probe.step(10)
    _, M, _, _ = probe.forces()
    inertia = abs(M[0, 2]) * 60 / (0.05 * om0)
    k_gen = 0.2 * abs(M[0, 2]) / om0 ** 2
    lat = P.Lattice.from_workload(wl)
    o = O.from_workload(wl)
    lat.set_drive(0, inertia, k_gen=k_gen)
    o.set_drive(0, inertia, k_gen=k_gen)
    rows = []
    for t in (10, 30, 60):
        lat.step(t - lat.t)
        o.step(t - o.t)
        thg, omg = lat.drive_state(0)
        tho, omo = o.drive_state(0)
        rows.append((t, omg, omo, thg - tho))
    print("t, Omega gpu, Omega oracle, dtheta:", rows)
    assert abs(rows[-1][2] / om0 - 1) > 0.01          # the rotor did change its speed
    for t, omg, omo, dth in rows:
        assert abs(omg - omo) <= 1e-5 * abs(omo), (t, omg, omo)
        assert abs(dth) <= 1e-6
    rg, ug = (a.cpu().numpy().astype(np.float64) for a in lat.fields())
    ro, uo = o.fields()
    assert _rel_l2(ug[:, 1:-1], uo[:, 1:-1]) <= 1e-5
    Fg, _ = lat.forces()
    Fo, _, _, _ = o.forces()
    assert np.abs(Fg - Fo).max() <= 1e-3 * np.abs(Fo).max()


def test_infinite_inertia_is_prescribed_rotation(P):
    wl = W.workload("rotor48")
    a = P.Lattice.from_workload(wl)
    b = P.Lattice.from_workload(wl)
    b.set_drive(0, 1e300)
    a.step(20)
    b.step(20)
    th, om = b.drive_state(0)
    om0 = wl.rotors[0].omega(wl.u_in)
    assert om == om0 and abs(th - 20 * om0) <= 1e-14
    ua, ub = (x.fields()[1].cpu().numpy().astype(np.float64) for x in (a, b))
    assert _rel_l2(ub, ua) <= 1e-6


def _no_blades():
    return BladeGrid(sdf=np.full((2, 2, 2), 100.0, np.float32), origin=(0.0, 0.0, 0.0), spacing=0.5,
                     radius=1.0, hub_radius=0.0, chord_root=1.0, chord_tip=1.0)


def test_sphere_spin_down_matches_oracle(P):
    """A sphere (radius 5, hub only) in a periodic 32^3 box of fluid at rest,
    spun for 200 steps, then released with an inertia that halves its speed
    in a few hundred steps."""
    om0, a, tau = 0.004, 5.0, 0.8
    lat = P.Lattice(32, 32, 32, open_boundaries=False, tau_mo=tau, c_smag=0.0, u_in=0.0, wall_model=False)
    lat.add_rotor(_no_blades(), center=(15.5, 15.5, 15.5), omega=om0, axis=2, n_blades=0, hub_radius=a)
    rot = O.make_rotor(_no_blades(), center=(15.5, 15.5, 15.5), axis=2, omega=om0, n_blades=0, hub_radius=a)
    o = O.Oracle(32, 32, 32, open_boundaries=False, tau_mo=tau, c_smag=0.0, u_in=0.0, wall_model=False,
                 rotors=[rot])
    lat.step(200)
    o.step(200)
    inertia = 3e5
    lat.set_drive(0, inertia)
    o.set_drive(0, inertia)
    lat.step(300)
    o.step(300)
    _, omg = lat.drive_state(0)
    _, omo = o.drive_state(0)
    assert omo < 0.8 * om0
    assert abs(omg - omo) <= 1e-5 * omo, (omg, omo)


def test_driven_snapshot_resume_and_gradient_refusal(P):
    wl = W.workload("rotor48")
    lat = P.Lattice.from_workload(wl)
    lat.set_drive(0, 1e3)
    lat.step(5)
    s = lat.save_state()
    lat.step(7)
    th1, om1 = lat.drive_state(0)
    u1 = lat.fields()[1].clone()
    lat.load_state(s)
    lat.step(7)
    th2, om2 = lat.drive_state(0)
    assert (th1, om1) == (th2, om2)
    import torch
    assert torch.equal(u1, lat.fields()[1])
    with pytest.raises(P.HlError) as e:
        lat.grad(4, 2, [1.0], [0.0], ckpt_every=2)
    assert e.value.code == -5


def test_convergence_study_workload_parity(P):
    """The finest-Reynolds-ladder workload of the grid-convergence study at its
    coarsest grid (R = 16, 64x64x128, tau = 0.50025, wall model on): fields
    against the FP64 oracle after 300 steps (relative L2 of rho and u <= 1e-5)
    and the rotor loads of every compared step (<= 1e-3)."""
    from paper_2510_13726_b300 import convergence as C
    wl = C.study_workload(16)
    assert abs(wl.tau_mo - 0.50025) < 1e-15
    lat = P.Lattice.from_workload(wl)
    o = O.from_workload(wl)
    for t_target in (100, 200, 300):
        lat.step(t_target - lat.t)
        o.step(t_target - o.t)
        rg, ug = (a.cpu().numpy().astype(np.float64) for a in lat.fields())
        ro, uo = o.fields()
        e_rho = np.linalg.norm((rg - ro)[1:-1]) / np.linalg.norm(ro[1:-1])
        e_u = np.linalg.norm((ug - uo)[:, 1:-1]) / np.linalg.norm(uo[:, 1:-1])
        Fg, _ = lat.forces()
        Mg, _ = lat.moments()
        Fo, Mo, _, _ = o.forces()
        eF = np.abs(Fg - Fo).max() / np.abs(Fo).max()
        eM = np.abs(Mg - Mo).max() / np.abs(Mo).max()
        print(f"R=16 study workload t={t_target}: rho {e_rho:.2e} u {e_u:.2e} F {eF:.2e} M {eM:.2e}")
        assert e_rho <= 1e-5 and e_u <= 1e-5, (t_target, e_rho, e_u)
        assert eF <= 1e-3 and eM <= 1e-3, (t_target, eF, eM)
    lat.close()


def test_convergence_study_driver(P):
    """The grid-convergence driver on three resolutions of each ladder (one
    revolution of spin-up, one averaged): the Reynolds ladder scales the
    viscosity with R, the y+ ladder keeps it, the interface ladder keeps it
    and scales the porosity transition with R; finite thrust coefficients and
    the derived orders and index."""
    from paper_2510_13726_b300 import convergence as C
    for ladder in ("reynolds", "yplus", "interface"):
        res = C.run_study(radii=(16, 32, 64), revolutions_spinup=1.0, revolutions_avg=1.0, ladder=ladder)
        rows = res["resolutions"]
        ct = [r["C_T"] for r in rows]
        assert all(np.isfinite(ct)) and all(c > 0 for c in ct)
        assert np.isfinite(res["apparent_order"]) and res["gci_finest"] >= 0.0
        taus = [r["tau"] for r in rows]
        if ladder in ("yplus", "interface"):
            assert taus == [0.5005] * 3
            assert rows[2]["Re"] == pytest.approx(4 * rows[0]["Re"])
            assert [r["eps_h"] for r in rows] == ([1.0, 2.0, 4.0] if ladder == "interface" else [2.0] * 3)
        else:
            assert taus[2] - 0.5 == pytest.approx(4 * (taus[0] - 0.5))
            assert rows[2]["Re"] == pytest.approx(rows[0]["Re"])
