"""Parity of the CUDA discrete adjoint (hl_grad) with the FP64 oracle's
adjoint, and of the forward extensions it relies on (static porosity
multiplier d0, frozen cell sets).

The oracle differentiates by complex step (pinned against finite
differences in test_oracle_adjoint.py); the CUDA path uses a hand-derived
FP32 vector-Jacobian product of the collision, a hand-derived reverse pass
of the wall model with FP64 forward-mode Newton derivatives, and FP32 pitch
tangents of the geometry.  Tolerances: FP32 rounding of the forward state
and of the adjoint arithmetic: 1e-4 relative on the gradients (observed
a few 1e-6).
"""

import numpy as np
import pytest

import oracle as O
import workloads as W

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


def _perm_to_oracle(q, P):
    c, _ = P.velocity_set(q)
    co, _, _ = O.lattice(q)
    idx = {tuple(v): i for i, v in enumerate(co)}
    return np.array([idx[tuple(v)] for v in c])


@pytest.mark.parametrize("q", [19, 27])
@pytest.mark.parametrize("branch", ["bulk", "band", "wall"])
def test_collision_vjp_unit_parity(P, q, branch):
    """hl_debug_collide_vjp against the oracle's complex-step VJP on 4096
    random cells (FP32 inputs seen exactly by both sides)."""
    import torch
    c, w = P.velocity_set(q)
    perm = _perm_to_oracle(q, P)
    inv = np.argsort(perm)
    n = 4096
    f = W.random_populations(31 + q, n, w, amplitude=0.1)
    g32 = (f - w).astype(np.float32)
    fin = w + g32.astype(np.float64)
    rng = np.random.default_rng(9)
    lam = rng.normal(0, 1, (n, q)).astype(np.float32)
    tau_mo, cs = 0.52, 0.1
    dev = "cuda"
    gin = torch.tensor(g32, device=dev)
    lin = torch.tensor(lam, device=dev)
    lout = torch.empty_like(lin)
    gd = torch.empty(n, device=dev)
    gu = torch.empty(n, 3, device=dev)
    gS = torch.empty(n, 6, device=dev)
    kw = {}
    if branch == "bulk":
        args = [0, 0, 0, 0]
    else:
        d = rng.uniform(0, 1, n).astype(np.float32)
        d[:256] = 0.0
        d[256:512] = 1.0
        uB = rng.uniform(-0.3, 0.3, (n, 3)).astype(np.float32)
        sig = (np.ones(n) if branch == "band" else np.zeros(n)).astype(np.float32)
        S6 = (rng.normal(size=(n, 6)) * 1e-3).astype(np.float32)
        td = [torch.tensor(a, device=dev).contiguous() for a in (d, uB, sig, S6)]
        args = [t.data_ptr() for t in td]
        S33 = np.zeros((n, 3, 3))
        for k, (a, b) in enumerate([(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]):
            S33[:, a, b] = S33[:, b, a] = S6[:, k]
        kw = dict(d=d.astype(np.float64), uB=uB.astype(np.float64), sigma=sig.astype(np.float64), Sfd=S33)
    rc = P.lib().hl_debug_collide_vjp(q, n, gin.data_ptr(), *args, tau_mo, cs, lin.data_ptr(), lout.data_ptr(),
                                      gd.data_ptr(), gu.data_ptr(), gS.data_ptr(),
                                      torch.cuda.current_stream().cuda_stream)
    assert rc == 0
    torch.cuda.synchronize()
    lf_o, gd_o, gu_o, gS_o = O.collide_vjp_cells(q, fin[:, inv], lam.astype(np.float64)[:, inv],
                                                 tau_mo=tau_mo, c_smag=cs, **kw)
    lf_o = lf_o[:, perm]
    lf = lout.cpu().numpy().astype(np.float64)
    scale = np.abs(lf_o).max()
    assert np.abs(lf - lf_o).max() <= 2e-5 * scale, np.abs(lf - lf_o).max() / scale
    gdg = gd.cpu().numpy().astype(np.float64)
    assert np.abs(gdg - gd_o).max() <= 2e-5 * max(1e-3, np.abs(gd_o).max())
    if branch != "bulk":
        gug = gu.cpu().numpy().astype(np.float64)
        assert np.abs(gug - gu_o).max() <= 2e-5 * max(1e-3, np.abs(gu_o).max())
        gSg = gS.cpu().numpy().astype(np.float64)
        want = np.stack([gS_o[:, 0, 0], gS_o[:, 1, 1], gS_o[:, 2, 2], gS_o[:, 0, 1] + gS_o[:, 1, 0],
                         gS_o[:, 0, 2] + gS_o[:, 2, 0], gS_o[:, 1, 2] + gS_o[:, 2, 1]], 1)
        assert np.abs(gSg - want).max() <= 2e-5 * max(1e-3, np.abs(want).max())


def _wl():
    return W.workload("rotor48_adj")


def _rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def test_forward_with_d0_and_frozen_sets_matches_oracle(P):
    """Forward extensions used by the gradient checks: a static porosity
    field d0 and a pitch change with the cell sets frozen."""
    import torch
    wl = _wl()
    rng = np.random.default_rng(3)
    d0 = 1.0 - 0.3 * rng.uniform(0, 1, (wl.nz, wl.ny, wl.nx))
    d0 = d0.astype(np.float32)
    lat = P.Lattice.from_workload(wl)
    o = O.from_workload(wl)
    lat.set_d0(torch.tensor(d0, device=lat.device))
    o.set_d0(d0.astype(np.float64))
    lat.freeze_sets(True)
    o.freeze_sets(True)
    lat.set_pitch(0, wl.rotors[0].pitch + 0.05)
    o.set_pitch(0, wl.rotors[0].pitch + 0.05)
    lat.step(12)
    o.step(12)
    rg, ug = (a.cpu().numpy().astype(np.float64) for a in lat.fields())
    ro, uo = o.fields()
    assert _rel_l2(ug[:, 1:-1], uo[:, 1:-1]) <= 1e-5
    assert np.linalg.norm((rg - ro)[1:-1]) / np.linalg.norm(ro[1:-1]) <= 1e-5
    Fg, _ = lat.forces()
    Fo, _, _, _ = o.forces()
    assert np.abs(Fg - Fo).max() <= 1e-3 * np.abs(Fo).max()


@pytest.mark.parametrize("wall_model", [True, False])
def test_gradient_parity_with_oracle(P, wall_model):
    """J, dJ/dpitch and dJ/dd0 of J = mean over the last 8 of 16 steps of
    thrust - 0.3 torque, checkpoints every 5 steps, against the oracle."""
    import torch
    wl = _wl()
    T, navg, wT, wQ = 16, 8, 1.0, -0.3
    lat = P.Lattice.from_workload(wl, wall_model=wall_model)
    Jg, gpg, gdg = lat.grad(T, navg, [wT], [wQ], ckpt_every=5)
    gdg = gdg.cpu().numpy().astype(np.float64)
    o = O.from_workload(wl, wall_model=wall_model)
    Jo, gpo, gdo = o.adjoint(T, navg, [wT], [wQ])
    print(f"J {Jg:.8e} vs {Jo:.8e}; dJ/dpitch {gpg[0]:.8e} vs {gpo[0]:.8e}; "
          f"dJ/dd0 rel L2 {_rel_l2(gdg, gdo):.2e}")
    # observed: J 4e-7, dJ/dpitch 5e-6, dJ/dd0 4e-6 (wall model on)
    assert abs(Jg - Jo) <= 1e-5 * abs(Jo)
    assert abs(gpg[0] - gpo[0]) <= 1e-4 * abs(gpo[0])
    assert _rel_l2(gdg, gdo) <= 1e-4
    # the lattice ends where hl_step(T) would leave it
    ref = P.Lattice.from_workload(wl, wall_model=wall_model)
    ref.step(T)
    r1, u1 = lat.fields()
    r2, u2 = ref.fields()
    assert torch.equal(r1, r2) and torch.equal(u1, u2)
    assert lat.t == T


def test_gradient_independent_of_checkpoint_spacing(P):
    """The segment recomputation reproduces the forward states: the gradient
    with a checkpoint every step, every 5 steps and one checkpoint agree."""
    wl = _wl()
    out = []
    for K in (1, 5, 16):
        lat = P.Lattice.from_workload(wl)
        J, gp, gd = lat.grad(16, 8, [1.0], [0.5], ckpt_every=K)
        out.append((J, gp[0], gd.cpu().numpy().astype(np.float64)))
    for J, gp, gd in out[1:]:
        assert J == out[0][0]
        assert abs(gp - out[0][1]) <= 1e-6 * abs(out[0][1])
        assert _rel_l2(gd, out[0][2]) <= 1e-6


def test_gradient_against_gpu_finite_differences(P):
    """dJ/dpitch against central differences of the CUDA forward itself
    (h = 1e-3 rad, cell sets frozen) and dJ/dd0 at cells around the rotor
    (h = 1e-2 on d0)."""
    import torch
    wl = _wl()
    T, navg, wT, wQ = 16, 8, 1.0, 0.5
    lat = P.Lattice.from_workload(wl)
    J0, gp, gd = lat.grad(T, navg, [wT], [wQ], ckpt_every=8)
    gd = gd.cpu().numpy()

    p0 = wl.rotors[0].pitch

    def J(pitch=0.0, d0=None):
        m = P.Lattice.from_workload(wl)
        if d0 is not None:
            m.set_d0(torch.tensor(d0, device=m.device))
        m.freeze_sets(True)
        m.set_pitch(0, p0 + pitch)
        m.step(T - navg)
        m.forces(reset_avg=True)
        m.step(navg)
        _, Fa = m.forces()
        _, Ma = m.moments()
        return wT * Fa[0, 2] + wQ * Ma[0, 2]

    h = 1e-3
    fd = (J(h) - J(-h)) / (2 * h)
    print("dJ/dpitch adjoint", gp[0], "FD", fd)
    assert abs(gp[0] - fd) <= 5e-3 * abs(fd)
    rng = np.random.default_rng(4)
    c = wl.rotors[0].center
    worst = 0.0
    for _ in range(6):
        cell = (int(c[2] + rng.integers(-6, 7)), int(c[1] + rng.integers(-12, 13)), int(c[0] + rng.integers(-12, 13)))
        e = np.ones((wl.nz, wl.ny, wl.nx), dtype=np.float32)
        hd = 1e-2
        e[cell] = 1.0 + hd
        Jp = J(d0=e)
        e[cell] = 1.0 - hd
        Jm = J(d0=e)
        fdd = (Jp - Jm) / (2 * hd)
        worst = max(worst, abs(gd[cell] - fdd) / max(abs(fdd), 1e-3 * abs(gp[0])))
    assert worst <= 2e-2, worst


def test_rotor_objective_autograd(P):
    """torch.autograd through rotor_objective equals hl_grad with the same weights."""
    import torch
    wl = _wl()
    lat = P.Lattice.from_workload(wl)
    pitch = torch.full((1,), wl.rotors[0].pitch, dtype=torch.float64, requires_grad=True)
    d0 = torch.ones(wl.nz, wl.ny, wl.nx, device=lat.device, requires_grad=True)
    T, Qv = P.rotor_objective(lat, pitch, d0, steps=12, avg_last=6, ckpt_every=4)
    (T.sum() - 0.2 * Qv.sum()).backward()
    ref = P.Lattice.from_workload(wl)
    ref.set_d0(torch.ones(wl.nz, wl.ny, wl.nx, device=ref.device))
    Jr, gpr, gdr = ref.grad(12, 6, [1.0], [-0.2], ckpt_every=4)
    assert abs(float((T[0] - 0.2 * Qv[0]).detach()) - Jr) <= 1e-9 * abs(Jr)
    assert abs(float(pitch.grad[0]) - gpr[0]) <= 1e-6 * abs(gpr[0])
    assert _rel_l2(d0.grad.cpu().numpy().astype(np.float64), gdr.cpu().numpy().astype(np.float64)) <= 1e-6


def test_wall_sample_outside_box_is_reported(P):
    """A blade grid without padding: a thin sheet (half a cell along T) whose
    signed distance is about 0.5 everywhere and rises along the axis, so the
    wall normals point axially and wall cells reach the axial edge of the
    rotor's reach.  Their velocity samples would leave the rotor box, which
    the second stream must not read: the step reports HL_ERR_GEOMETRY and
    leaves those cells unmodelled."""
    import dataclasses
    wl = _wl()
    g0 = wl.blade_grids()[0]
    gx = g0.sdf.shape[2]
    gz = 17
    sdf = 0.5 + 1e-3 * np.arange(gz, dtype=np.float32)[:, None, None] + np.zeros((gz, 2, gx), np.float32)
    grid = dataclasses.replace(g0, sdf=np.ascontiguousarray(sdf, dtype=np.float32),
                               origin=(g0.origin[0], -0.25, -4.0))
    # sample 4 cells off the wall: from the axial edge of the reach (3 cells
    # off the centre plane) the trilinear corners reach 8 cells, the box 7
    lat = P.Lattice(wl.nx, wl.ny, wl.nz, wm_ysample=4.0)
    spec = wl.rotors[0]
    lat.add_rotor(grid, center=spec.center, omega=spec.omega(wl.u_in))
    with pytest.raises(P.HlError) as e:
        lat.step(1)
    assert e.value.code == -9


def test_gradient_study_128x128x256_against_finite_differences(P):
    """The gradient study (128x128x256 D3Q19, R = 32, wall model on): mean
    thrust over the last 1000 of 4000 steps, checkpoint every 100 steps,
    against central differences of the CUDA forward (cell sets frozen; J is
    the FP64 running mean of the per-step FP64 force sums).

    Step sizes from an h-sweep of this workload: the pitch difference falls
    onto the adjoint as h shrinks (relative gap 1.1e-2 at h = 1e-3, 2.0e-3 at
    1e-4, 2.6e-4 at 3e-5: the trilinear blade grid's kinks make J only
    piecewise smooth in the pitch) until the forward's rounding noise, which
    grows like 1/h, takes over (at h = 1e-5 one run gave 3.6e-5, another
    9.7e-4 on rounding-level changes of the collision).  The test holds the
    adjoint to D(3e-5) within 1e-3, or within twice the noise measured as
    |D(3e-5) - D(3.3e-5)| if that is larger.  A single cell's d0 moves J by ~1e-4 per unit,
    so its difference carries the forward's rounding noise: the median error
    over the 32 cells follows n/h + c h^2 (n ~ 6e-6, c ~ 7; 6.1e-3 at h =
    0.03, 1.4e-3 at 0.01, 2.7e-3 at 0.003, 5.7e-3 at 0.001).  The test takes
    the Richardson extrapolation (4 D(h/2) - D(h)) / 3 from h = 0.02 and 0.01,
    which removes the h^2 term, and measures the noise itself as the spread
    of two nearby differences, D(0.01) and D(0.0105), whose truncation is the
    same to 1e-4: the median relative error must be within 1e-3 or within
    twice the median noise level, whichever is larger."""
    import torch
    wl = W.workload("rotor128_adj")
    T, navg, K = 4000, 1000, 100
    lat = P.Lattice.from_workload(wl)
    s0 = lat.save_state()
    J, gp, gd = lat.grad(T, navg, [1.0], [0.0], ckpt_every=K)
    gd = gd.cpu().numpy()
    p0 = wl.rotors[0].pitch

    def Jrun(dp=0.0, d0=None):
        lat.load_state(s0)
        lat.set_d0(None if d0 is None else torch.tensor(d0, device=lat.device))
        lat.freeze_sets(True)
        lat.set_pitch(0, p0 + dp)
        lat.step(T - navg)
        lat.forces(reset_avg=True)
        lat.step(navg)
        _, Fa = lat.forces()
        lat.freeze_sets(False)
        lat.set_pitch(0, p0)
        return Fa[0, wl.flow_axis]

    assert abs(Jrun() - J) <= 1e-12 * abs(J)
    fd = {h: (Jrun(h) - Jrun(-h)) / (2 * h) for h in (1e-4, 3.3e-5, 3e-5, 1e-5)}
    print("dJ/dpitch adjoint %.7f; central differences %s" % (gp[0], {h: round(v, 7) for h, v in fd.items()}))
    noise_p = abs(fd[3e-5] - fd[3.3e-5]) / abs(fd[3e-5])
    assert abs(gp[0] - fd[3e-5]) <= max(1e-3, 2 * noise_p) * abs(fd[3e-5])
    rng = np.random.default_rng(11)
    c, R = wl.rotors[0].center, wl.rotors[0].radius
    cells = []
    while len(cells) < 32:
        off = rng.uniform(-2 * R, 2 * R, 3)
        if np.linalg.norm(off) <= 2 * R:
            x, y, z = (int(round(c[k] + off[k])) for k in range(3))
            cells.append((z, y, x))

    def D(cell, h):
        e = np.ones((wl.nz, wl.ny, wl.nx), np.float32)
        e[cell] = 1.0 + h
        Jp = Jrun(d0=e)
        e[cell] = 1.0 - h
        return (Jp - Jrun(d0=e)) / (2 * h)

    adj, rich, spread = [], [], []
    for cell in cells:
        d1, d2, d3 = D(cell, 0.02), D(cell, 0.01), D(cell, 0.0105)
        adj.append(float(gd[cell]))
        rich.append((4 * d2 - d1) / 3)
        spread.append(abs(d2 - d3))
    adj, rich, spread = np.array(adj), np.array(rich), np.array(spread)
    scale = np.abs(rich).max()
    den = np.maximum(np.abs(rich), 0.05 * scale)
    rel = np.abs(adj - rich) / den
    noise = spread / den
    print("dJ/dd0 (Richardson h = 0.02/0.01) relative error: median %.3g, 90th percentile %.3g, max %.3g; "
          "noise (|D(0.01) - D(0.0105)|) median %.3g" % (np.median(rel), np.percentile(rel, 90), rel.max(),
                                                         np.median(noise)))
    assert np.median(rel) <= max(1e-3, 2 * np.median(noise))
    assert np.percentile(rel, 90) <= max(1e-2, 4 * np.percentile(noise, 90))


def test_gradient_with_held_caller_inflow_plane(P):
    """hl_grad with a caller's inflow plane (held at its content for the
    sweep: forward pass, recompute and reverse all see it).  A plane equal to
    the uniform synthetic inflow reproduces the synthetic sweep; a sheared
    plane (axial velocity u_in (1 + 0.3 sin(2 pi y / n_y))) gives the
    forward's objective and a pitch gradient that matches central differences
    of the CUDA forward run with the same plane (h = 1e-3 rad, cell sets
    frozen)."""
    import torch
    from workloads.configs import Workload, _single
    wl = Workload("plane48", 48, 48, 64, turbulence=0.0, rotors=_single(48, 48, 64, 12.0, 6.0))
    T, navg, wT, wQ = 48, 8, 1.0, 0.5     # the inlet's signal reaches the rotor (16 cells downstream)

    def plane_of(lat, shear):
        n_c, n_b = lat.inflow_plane_shape()[1:]
        pl = torch.zeros(lat.inflow_plane_shape(), dtype=torch.float32)
        prof = 1.0 + shear * torch.sin(2 * np.pi * torch.arange(n_c, dtype=torch.float64) / n_c)
        pl[wl.flow_axis] = (wl.u_in * prof)[:, None].float().expand(n_c, n_b)
        return pl.to(lat.device)

    ref = P.Lattice.from_workload(wl)
    Jr, gpr, gdr = ref.grad(T, navg, [wT], [wQ], ckpt_every=8)
    lat = P.Lattice.from_workload(wl)
    uniform = plane_of(lat, 0.0)
    lat.set_inflow_plane(uniform)
    Ju, gpu_, gdu = lat.grad(T, navg, [wT], [wQ], ckpt_every=8)
    assert abs(Ju - Jr) <= 1e-12 * abs(Jr)
    assert abs(gpu_[0] - gpr[0]) <= 1e-6 * abs(gpr[0])
    assert _rel_l2(gdu.double().cpu().numpy(), gdr.double().cpu().numpy()) <= 1e-6
    lat.close()
    ref.close()

    p0 = wl.rotors[0].pitch
    lat = P.Lattice.from_workload(wl)
    sheared = plane_of(lat, 0.3)
    lat.set_inflow_plane(sheared)
    Js, gps, _ = lat.grad(T, navg, [wT], [wQ], ckpt_every=8)
    lat.close()
    assert abs(Js - Jr) > 1e-3 * abs(Jr)          # the plane changes the flow

    def J(pitch):
        m = P.Lattice.from_workload(wl)
        m.set_inflow_plane(sheared)
        m.freeze_sets(True)
        m.set_pitch(0, p0 + pitch)
        m.step(T - navg)
        m.forces(reset_avg=True)
        m.step(navg)
        _, Fa = m.forces()
        _, Ma = m.moments()
        m.close()
        return wT * Fa[0, 2] + wQ * Ma[0, 2]

    assert abs(J(0.0) - Js) <= 1e-9 * abs(Js)     # the sweep's forward pass ran on the plane
    h = 1e-3
    fd = (J(h) - J(-h)) / (2 * h)
    print("sheared plane: dJ/dpitch adjoint", gps[0], "FD", fd)
    # observed 3.8e-3 (FP32 forward differences over 48 steps; blade-grid
    # kinks crossed within +-h); a sweep linearised about the synthetic
    # inflow instead of the plane is off by far more
    assert abs(gps[0] - fd) <= 1e-2 * abs(fd)
    print("synthetic-inflow sweep dJ/dpitch", gpr[0])
    assert abs(gpr[0] - fd) > 3e-2 * abs(fd)


def test_gradient_parity_two_rotors(P):
    """Two rotors in tandem with their own objective weights (the second in
    the first's wake, other tip-speed ratio, phase and pitch): J, dJ/dpitch
    of each rotor and dJ/dd0 against the oracle's adjoint."""
    from workloads.configs import RotorSpec, Workload
    wl = Workload("two48", 48, 48, 128, turbulence=0.05,
                  rotors=[RotorSpec(center=(23.5, 23.5, 32.0), radius=10.0, tsr=6.0),
                          RotorSpec(center=(23.5, 23.5, 88.0), radius=10.0, tsr=5.0, phase0=0.7, pitch=0.05)])
    T, navg = 16, 8
    wT, wQ = [1.0, 0.5], [-0.3, 0.2]
    lat = P.Lattice.from_workload(wl)
    Jg, gpg, gdg = lat.grad(T, navg, wT, wQ, ckpt_every=5)
    gdg = gdg.cpu().numpy().astype(np.float64)
    o = O.from_workload(wl)
    Jo, gpo, gdo = o.adjoint(T, navg, wT, wQ)
    print(f"two rotors: J {Jg:.8e} vs {Jo:.8e}; dJ/dpitch {list(gpg)} vs {list(gpo)}; "
          f"dJ/dd0 rel L2 {_rel_l2(gdg, gdo):.2e}")
    assert abs(Jg - Jo) <= 1e-5 * abs(Jo)
    for k in range(2):
        assert abs(gpg[k] - gpo[k]) <= 1e-4 * abs(gpo[k]), k
    assert _rel_l2(gdg, gdo) <= 1e-4


def test_gradient_through_a_collapsed_friction_velocity(P):
    """A hub wall cell of the off-centre second rotor carries a friction
    velocity of ~4e-7 from step to step (warm starts; |u_t| ~ 6e-4 near the
    axis), so u+ ~ 1700: exp(kappa u+) ~ 1e304 and the Newton derivative f'
    overflows to -inf, and the step is 0; its dual-number derivative must be
    0 too (the quotient rule gave 0 * inf = NaN and poisoned the whole
    gradient).  Gradients
    are finite and match the oracle (complex division by an infinite value
    also gives 0): pitch to 1e-4, dJ/dd0 to the 1e-3 gradient tolerance
    (observed 7.5e-4: the cells around the collapsed one carry it, the
    rest agree to 2e-4)."""
    from workloads.configs import RotorSpec, Workload
    wl = Workload("hub48", 48, 48, 128, turbulence=0.05,
                  rotors=[RotorSpec(center=(23.5, 23.5, 32.0), radius=10.0, tsr=6.0),
                          RotorSpec(center=(24.0, 23.0, 88.0), radius=10.0, tsr=5.0, phase0=0.7, pitch=0.05)])
    T, navg = 16, 8
    wT, wQ = [1.0, 0.5], [-0.3, 0.2]
    lat = P.Lattice.from_workload(wl)
    Jg, gpg, gdg = lat.grad(T, navg, wT, wQ, ckpt_every=5)
    gdg = gdg.cpu().numpy().astype(np.float64)
    assert np.isfinite(gpg).all() and np.isfinite(gdg).all()
    o = O.from_workload(wl)
    Jo, gpo, gdo = o.adjoint(T, navg, wT, wQ)
    print(f"collapsed u_tau: dJ/dpitch {list(gpg)} vs {list(gpo)}; dJ/dd0 rel L2 {_rel_l2(gdg, gdo):.2e}")
    for k in range(2):
        assert abs(gpg[k] - gpo[k]) <= 1e-4 * abs(gpo[k]), k
    assert _rel_l2(gdg, gdo) <= 1e-3


def test_gradient_parity_d3q27(P):
    """The gradient sweep on D3Q27 (the third-order H_xyz term enters the
    collision VJP; 27-slot gathers in every reverse kernel) against the
    oracle's adjoint on the same lattice."""
    wl = _wl()
    wl.q = 27
    T, navg, wT, wQ = 16, 8, 1.0, -0.3
    lat = P.Lattice.from_workload(wl)
    Jg, gpg, gdg = lat.grad(T, navg, [wT], [wQ], ckpt_every=5)
    gdg = gdg.cpu().numpy().astype(np.float64)
    o = O.from_workload(wl)
    Jo, gpo, gdo = o.adjoint(T, navg, [wT], [wQ])
    print(f"D3Q27: J {Jg:.8e} vs {Jo:.8e}; dJ/dpitch {gpg[0]:.8e} vs {gpo[0]:.8e}; "
          f"dJ/dd0 rel L2 {_rel_l2(gdg, gdo):.2e}")
    assert abs(Jg - Jo) <= 1e-5 * abs(Jo)
    assert abs(gpg[0] - gpo[0]) <= 1e-4 * abs(gpo[0])
    assert _rel_l2(gdg, gdo) <= 1e-4


@pytest.mark.parametrize("storage", ["f16s", "bf16s"])
def test_gradient_with_16bit_storage(P, storage):
    """The sweep with populations stored in 16 bits (checkpoints and
    recomputed states in the same storage, FP32 arithmetic) against the
    FP64 oracle: the storage rounding of each step enters the trajectory,
    so the objective and gradients agree to the storage precision, not to
    FP32."""
    wl = _wl()
    T, navg, wT, wQ = 16, 8, 1.0, -0.3
    lat = P.Lattice.from_workload(wl, storage=storage)
    Jg, gpg, gdg = lat.grad(T, navg, [wT], [wQ], ckpt_every=5)
    gdg = gdg.cpu().numpy().astype(np.float64)
    o = O.from_workload(wl)
    Jo, gpo, gdo = o.adjoint(T, navg, [wT], [wQ])
    print(f"{storage}: J {Jg:.8e} vs {Jo:.8e}; dJ/dpitch {gpg[0]:.8e} vs {gpo[0]:.8e}; "
          f"dJ/dd0 rel L2 {_rel_l2(gdg, gdo):.2e}")
    # observed: J 7e-5 / 4e-5, dJ/dpitch 3e-4 / 2.2e-3, dJ/dd0 3.5e-4 / 1.4e-3 (FP16 / BF16)
    assert np.isfinite(gdg).all()
    assert abs(Jg - Jo) <= 5e-4 * abs(Jo)
    assert abs(gpg[0] - gpo[0]) <= 1e-2 * abs(gpo[0])
    assert _rel_l2(gdg, gdo) <= 1e-2
