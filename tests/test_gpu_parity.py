"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (FP32 arithmetic, weight-shifted FP32 storage):
  * single-cell collision: |f*_gpu - f*_oracle| <= 2e-6 w_i, the oracle fed
    the exact binary32 inputs the kernel sees (a few dozen FP32 roundings of
    quantities of size <= 0.3 w_i);
  * geometry: the binary32 decision value is evaluated in the same operation
    order on both sides, so the cell sets (force cells, wall cells) match
    bit for bit and the porosity to FP32 rounding;
  * whole-lattice fields: relative L2 error of density and velocity <= 1e-5
    after 200 steps (the accuracy target for FP32 storage), taken over the
    cells that are not on an open boundary plane.
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


def _rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


@pytest.mark.parametrize("q", [19, 27])
@pytest.mark.parametrize("branch", ["bulk", "band", "wall"])
def test_collision_unit_parity(P, q, branch):
    import torch
    c, w = P.velocity_set(q)
    perm = _perm_to_oracle(q, P)           # gpu slot s -> oracle index perm[s]
    n = 8192
    f = W.random_populations(21 + q, n, w, amplitude=0.1)
    g32 = (f - w).astype(np.float32)
    fin = w + g32.astype(np.float64)       # exactly what the kernel sees
    rng = np.random.default_rng(5)
    tau_mo, cs = 0.52, 0.1
    dev = "cuda"
    gin = torch.tensor(g32, device=dev)
    gout = torch.empty_like(gin)
    if branch == "bulk":
        args = [0, 0, 0, 0]
        d = uB = sig = S = None
    else:
        d = rng.uniform(0, 1, n).astype(np.float32)
        d[:512] = 0.0
        d[512:1024] = 1.0
        uB = rng.uniform(-0.3, 0.3, (n, 3)).astype(np.float32)
        sig = (np.ones(n) if branch == "band" else np.zeros(n)).astype(np.float32)
        S6 = (rng.normal(size=(n, 6)) * 1e-3).astype(np.float32)
        S = S6
        td = [torch.tensor(a, device=dev).contiguous() for a in (d, uB, sig, S6)]
        args = [t.data_ptr() for t in td]
    lib = P.lib()
    rc = lib.hl_debug_collide(q, n, gin.data_ptr(), *args, tau_mo, cs, gout.data_ptr(),
                              torch.cuda.current_stream().cuda_stream)
    assert rc == 0
    torch.cuda.synchronize()
    fgpu = gout.cpu().numpy().astype(np.float64) + w
    inv = np.argsort(perm)
    kw = {}
    if branch != "bulk":
        S33 = np.zeros((n, 3, 3))
        idx = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]
        for k, (a, b) in enumerate(idx):
            S33[:, a, b] = S33[:, b, a] = S[:, k]
        kw = dict(d=d.astype(np.float64), uB=uB.astype(np.float64), sigma=sig.astype(np.float64), Sfd=S33)
    # oracle in its own slot order: column j of the oracle holds gpu slot inv[j]
    fo, _ = O.collide_cells(q, fin[:, inv], tau_mo=tau_mo, c_smag=cs, **kw)
    fo = fo[:, perm]
    err = np.abs(fgpu - fo) / w
    assert err.max() <= 2e-6, err.max()


@pytest.mark.parametrize("q", [19, 27])
def test_packed_collision_unit_parity(P, q):
    """The packed two-cell bulk collision (FP32x2) against the oracle's
    single-cell collision (2e-6 w_i, as the one-cell kernel) and against the
    one-cell kernel itself (a few FP32 roundings), on random states and on
    equilibrium-like states of fast flows (|u| up to 0.15)."""
    import torch
    c, w = P.velocity_set(q)
    perm = _perm_to_oracle(q, P)
    n = 8192
    f = W.random_populations(31 + q, n, w, amplitude=0.1)
    rng = np.random.default_rng(9)
    u = rng.uniform(-0.15, 0.15, (n // 2, 3))
    cu = u @ np.asarray(c, dtype=np.float64).T
    feq = w * (1 + 3 * cu + 4.5 * cu ** 2 - 1.5 * (u ** 2).sum(1, keepdims=True))
    f[n // 2:] = feq * (1 + 0.02 * rng.uniform(-1, 1, feq.shape))
    g32 = (f - w).astype(np.float32)
    fin = w + g32.astype(np.float64)
    tau_mo, cs = 0.5005, 0.1
    gin = torch.tensor(g32, device="cuda")
    gp = torch.empty_like(gin)
    gs = torch.empty_like(gin)
    lib = P.lib()
    st = torch.cuda.current_stream().cuda_stream
    assert lib.hl_debug_collide_pair(q, n, gin.data_ptr(), tau_mo, cs, gp.data_ptr(), st) == 0
    assert lib.hl_debug_collide(q, n, gin.data_ptr(), 0, 0, 0, 0, tau_mo, cs, gs.data_ptr(), st) == 0
    assert lib.hl_debug_collide_pair(q, 3, gin.data_ptr(), tau_mo, cs, gp.data_ptr(), st) == -1   # n odd
    torch.cuda.synchronize()
    fpair = gp.cpu().numpy().astype(np.float64) + w
    fone = gs.cpu().numpy().astype(np.float64) + w
    inv = np.argsort(perm)
    fo, _ = O.collide_cells(q, fin[:, inv], tau_mo=tau_mo, c_smag=cs)
    fo = fo[:, perm]
    err = np.abs(fpair - fo) / w
    assert err.max() <= 2e-6, err.max()
    assert (np.abs(fpair - fone) / w).max() <= 1e-6


def _wl48():
    return W.workload("rotor48")


def test_geometry_sets_bit_exact(P):
    """Force-cell and wall-cell sets of the embedding agree bit for bit with
    the oracle at several rotor angles; porosity to FP32 rounding."""
    wl = _wl48()
    lat = P.Lattice.from_workload(wl)
    o = O.from_workload(wl)
    for t_target in (1, 2, 37):
        lat.step(t_target - lat.t)
        o.step(t_target - o.t)
        band = lat.rotor_band(0)
        lo, n = band["lo"], band["n"]
        _, d_or, fl_or, _ = o.geometry()
        sl = (slice(lo[2], lo[2] + n[2]), slice(lo[1], lo[1] + n[1]), slice(lo[0], lo[0] + n[0]))
        fl_gpu = band["flags"].cpu().numpy()
        assert np.array_equal(fl_gpu, fl_or[sl]), (t_target, np.argwhere(fl_gpu != fl_or[sl])[:5])
        outside = fl_or.copy()
        outside[sl] = 0
        assert not outside.any()
        assert np.abs(band["d"].cpu().numpy() - d_or[sl]).max() < 2e-6
        assert (fl_gpu & 2).sum() > 50


def test_wall_model_outputs(P):
    """Wall-model velocity and strain on the wall cells after the first steps."""
    wl = _wl48()
    lat = P.Lattice.from_workload(wl)
    o = O.from_workload(wl)
    for t_target in (1, 5):
        lat.step(t_target - lat.t)
        o.step(t_target - o.t)
        band = lat.rotor_band(0)
        lo, n = band["lo"], band["n"]
        du, S, ut, act, _ = o.wall_state()
        sl = (slice(lo[2], lo[2] + n[2]), slice(lo[1], lo[1] + n[1]), slice(lo[0], lo[0] + n[0]))
        wall = (band["flags"].cpu().numpy() & 2) > 0
        wm = band["wm"].cpu().numpy()
        du_g = np.stack([wm[0], wm[1], wm[2]], -1)[wall]
        du_o = du[sl][wall]
        scale = np.abs(du_o).max()
        assert np.abs(du_g - du_o).max() < 1e-4 * scale
        S_o = S[sl][wall]
        S_g = np.stack([wm[3], wm[4], wm[5], wm[6], wm[7], wm[8]], -1)[wall]
        S_o6 = np.stack([S_o[:, 0, 0], S_o[:, 1, 1], S_o[:, 2, 2], S_o[:, 0, 1], S_o[:, 0, 2], S_o[:, 1, 2]], -1)
        assert np.abs(S_g - S_o6).max() < 1e-4 * np.abs(S_o6).max()
        assert np.abs(band["utau"].cpu().numpy()[wall] - ut[sl][wall]).max() < 1e-4 * ut[sl][wall].max()


def _interior(a, axis_from_end=True):
    return a[..., 1:-1, :, :] if axis_from_end else a


def test_whole_step_parity_rotor48(P):
    """The 48x48x96 rotor (D3Q19, uniform inflow, R = 12, TSR 6, wall model,
    C_S = 0.1, tau_mo = 0.5005): fields and forces over 200 steps."""
    wl = _wl48()
    lat = P.Lattice.from_workload(wl)
    o = O.from_workload(wl)
    report = []
    for t_target in (1, 10, 50, 100, 150, 200):
        lat.step(t_target - lat.t)
        o.step(t_target - o.t)
        rg, ug = (a.cpu().numpy().astype(np.float64) for a in lat.fields())
        ro, uo = o.fields()
        er = _rel_l2(rg[1:-1] - 1.0, ro[1:-1] - 1.0)
        e_rho = np.linalg.norm((rg - ro)[1:-1]) / np.linalg.norm(ro[1:-1])
        e_u = _rel_l2(ug[:, 1:-1], uo[:, 1:-1])
        Fg, _ = lat.forces()
        Mg, _ = lat.moments()
        Fo, Mo, _, _ = o.forces()
        eF = np.abs(Fg - Fo).max() / np.abs(Fo).max()
        eM = np.abs(Mg - Mo).max() / np.abs(Mo).max()
        report.append((t_target, e_rho, e_u, er, eF, eM))
    print("t, rel L2 rho, rel L2 u, rel L2 (rho-1), F, M:", report)
    t, e_rho, e_u, er, eF, eM = report[-1]
    assert e_rho <= 1e-5 and e_u <= 1e-5, report
    for row in report:
        assert row[1] <= 1e-5 and row[2] <= 1e-5, row
        assert row[4] <= 1e-3 and row[5] <= 1e-3, row


def test_taylor_green_periodic(P):
    """Periodic Taylor-Green vortex (no rotor, C_S = 0): fields against the
    oracle and the analytic viscous decay."""
    import math
    import torch
    n, nz, tau, U0 = 32, 4, 0.8, 0.01
    k = 2 * math.pi / n
    Z, Y, X = np.meshgrid(np.arange(nz), np.arange(n), np.arange(n), indexing="ij")
    ux = -U0 * np.cos(k * X) * np.sin(k * Y)
    uy = U0 * np.sin(k * X) * np.cos(k * Y)
    rho = 1 - 3 * U0**2 / 4 * (np.cos(2 * k * X) + np.cos(2 * k * Y))
    u = np.stack([ux, uy, 0 * ux])
    lat = P.Lattice(n, n, nz, open_boundaries=False, tau_mo=tau, c_smag=0.0, u_in=0.0, wall_model=False)
    rho32, u32 = rho.astype(np.float32), u.astype(np.float32)
    lat.init_fields(torch.tensor(rho32.ravel()), torch.tensor(u32.reshape(3, -1)))
    o = O.Oracle(n, n, nz, open_boundaries=False, tau_mo=tau, c_smag=0.0, u_in=0.0, wall_model=False)
    o.init_equilibrium(rho32.astype(np.float64), u32.astype(np.float64))
    lat.step(250)
    o.step(250)
    rg, ug = (a.cpu().numpy().astype(np.float64) for a in lat.fields())
    ro, uo = o.fields()
    assert _rel_l2(ug, uo) <= 1e-5
    assert np.abs(rg - ro).max() <= 1e-6


def test_turbulent_inflow_channel(P):
    """Open channel with synthetic turbulent inflow and equilibrium outlet (no rotor)."""
    modes = W.fourier_modes(7, 32, 64.0, 0.05, 0.05)
    kw = dict(tau_mo=0.52, c_smag=0.1, u_in=0.05, wall_model=False)
    lat = P.Lattice(24, 20, 64, modes=modes, **kw)
    o = O.Oracle(24, 20, 64, modes=modes, **kw)
    lat.step(80)
    o.step(80)
    rg, ug = (a.cpu().numpy().astype(np.float64) for a in lat.fields())
    ro, uo = o.fields()
    assert _rel_l2(ug[:, 1:-1], uo[:, 1:-1]) <= 1e-5
    assert np.linalg.norm((rg - ro)[1:-1]) / np.linalg.norm(ro[1:-1]) <= 1e-5


def test_checkpoint_resume_is_bit_exact(P):
    import torch
    wl = _wl48()
    lat = P.Lattice.from_workload(wl)
    lat.step(5)
    snap = lat.save_state()
    lat.step(7)
    ra, ua = lat.fields()
    Fa, Fa_avg = lat.forces()
    lat.load_state(snap)
    assert lat.t == 5
    lat.step(7)
    rb, ub = lat.fields()
    Fb, Fb_avg = lat.forces()
    assert torch.equal(ra, rb) and torch.equal(ua, ub)
    # the order of the FP64 force sum follows the atomic fill order of the
    # force-cell list, so forces agree to FP64 rounding rather than bit for bit
    assert np.allclose(Fa, Fb, rtol=1e-12, atol=0) and np.allclose(Fa_avg, Fb_avg, rtol=1e-12, atol=0)


def test_nonfinite_state_is_reported_not_trapped(P):
    """A NaN seeded into the density makes hl_step return HL_ERR_NONFINITE
    through the device error word; the context stays usable."""
    import torch
    lat = P.Lattice(16, 16, 16, open_boundaries=False, u_in=0.0, wall_model=False)
    rho = torch.ones(16 ** 3)
    rho[1234] = float("nan")
    lat.init_fields(rho, None)
    with pytest.raises(P.HlError) as e:
        lat.step(2)
    assert e.value.code == -3
    lat.init_fields(torch.ones(16 ** 3), None)
    lat.step(2)


def test_mass_conservation_periodic_rotor(P):
    g = W.make_blade_grid(12.0)
    lat = P.Lattice(48, 48, 48, open_boundaries=False, wall_model=True, mass_check_every=10, mass_tol=1e-5)
    lat.add_rotor(g, center=(23.5, 23.5, 24.0), omega=0.025)
    m0 = lat.mass()
    lat.step(100)
    assert abs(lat.mass() - m0) / m0 < 1e-6


def test_overlap_schedule_is_bit_identical(P):
    """The two-stream schedule (bulk cells on the lattice stream, rotor-box
    chain on the internal stream) computes exactly what one stream computes."""
    import torch
    wl = _wl48()
    a = P.Lattice.from_workload(wl, overlap=True)
    b = P.Lattice.from_workload(wl, overlap=False)
    a.step(37)
    b.step(37)
    ra, ua = a.fields()
    rb, ub = b.fields()
    assert torch.equal(ra, rb) and torch.equal(ua, ub)
    Fa, Faa = a.forces()
    Fb, Fba = b.forces()
    assert np.allclose(Fa, Fb, rtol=1e-12, atol=0) and np.allclose(Faa, Fba, rtol=1e-12, atol=0)
    a.step(1)
    b.step(1)
    assert torch.equal(a.fields()[1], b.fields()[1])


def test_d3q27_whole_step_parity(P):
    """D3Q27 (adds the H_xyz third-order term) on the 48x48x96 rotor, FP32
    storage: fields after 200 steps within the FP32 tolerance."""
    wl = _wl48()
    wl.q = 27
    lat = P.Lattice.from_workload(wl)
    o = O.from_workload(wl)
    for t_target in (1, 50, 200):
        lat.step(t_target - lat.t)
        o.step(t_target - o.t)
        rg, ug = (a.cpu().numpy().astype(np.float64) for a in lat.fields())
        ro, uo = o.fields()
        e_rho = np.linalg.norm((rg - ro)[1:-1]) / np.linalg.norm(ro[1:-1])
        e_u = _rel_l2(ug[:, 1:-1], uo[:, 1:-1])
        assert e_rho <= 1e-5 and e_u <= 1e-5, (t_target, e_rho, e_u)
    Fg, _ = lat.forces()
    Fo, _, _, _ = o.forces()
    assert np.abs(Fg - Fo).max() <= 1e-3 * np.abs(Fo).max()


@pytest.mark.parametrize("storage", ["f16s", "bf16s"])
def test_16bit_storage_rotor48(P, storage):
    """16-bit population storage (f_i - w_i in FP16 / BF16, FP32 arithmetic) on
    the 48x48x96 rotor: time-averaged thrust and torque over steps 101-200
    within 1 % of the FP64 oracle (the 16-bit accuracy target)."""
    wl = _wl48()
    lat = P.Lattice.from_workload(wl, storage=storage)
    o = O.from_workload(wl)
    lat.step(100)
    o.step(100)
    lat.forces(reset_avg=True)
    o.reset_average()
    lat.step(100)
    o.step(100)
    _, Fa = lat.forces()
    _, Ma = lat.moments()
    _, _, Fo, Mo = o.forces()
    a = wl.flow_axis
    assert abs(Fa[0, a] - Fo[0, a]) <= 0.01 * abs(Fo[0, a]), (Fa, Fo)
    assert abs(Ma[0, a] - Mo[0, a]) <= 0.01 * abs(Mo[0, a]), (Ma, Mo)


def test_16bit_precision_study_rotor256_q27(P):
    """The precision study: D3Q27 128x128x256 rotor (R = 32, TSR 7), 1000 steps,
    thrust and torque averaged over the last 500 steps, FP32 / FP16 / BF16
    storage against the stored FP64 oracle run (tests/golden)."""
    import json
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "precision_rotor256_q27.json")
    ref = json.load(open(path))
    wl = W.workload("rotor256_q27")
    a = wl.flow_axis
    out = {}
    for storage in ("f32", "f16s", "bf16s"):
        lat = P.Lattice.from_workload(wl, storage=storage)
        lat.step(ref["average_from_step"])
        lat.forces(reset_avg=True)
        lat.step(ref["steps"] - ref["average_from_step"])
        _, Fa = lat.forces()
        _, Ma = lat.moments()
        out[storage] = (abs(Fa[0, a] / ref["thrust_mean"] - 1), abs(Ma[0, a] / ref["torque_mean"] - 1))
        lat.close()
    print("relative error of mean thrust, torque:", out)
    assert out["f32"][0] < 1e-3 and out["f32"][1] < 1e-3
    for s in ("f16s", "bf16s"):
        assert out[s][0] <= 0.01 and out[s][1] <= 0.01, (s, out[s])


def _parity_run(P, wl, checkpoints):
    lat = P.Lattice.from_workload(wl)
    o = O.from_workload(wl)
    rows = []
    for t_target in checkpoints:
        lat.step(t_target - lat.t)
        o.step(t_target - o.t)
        rg, ug = (a.cpu().numpy().astype(np.float64) for a in lat.fields())
        ro, uo = o.fields()
        a = wl.flow_axis
        inner = [slice(None)] * 3
        inner[2 - a] = slice(1, -1)          # fields are (nz, ny, nx): drop the open planes
        inner = tuple(inner)
        e_rho = float(np.linalg.norm((rg - ro)[inner]) / np.linalg.norm(ro[inner]))
        e_u = _rel_l2(ug[(slice(None),) + inner], uo[(slice(None),) + inner])
        rows.append((t_target, e_rho, e_u))
    Fg, _ = lat.forces()
    Fo, _, _, _ = o.forces()
    return rows, float(np.abs(Fg - Fo).max() / np.abs(Fo).max())


def test_flow_along_x_parity(P):
    """Rotor and inflow along x (96x48x48, R = 12, TSR 6, 5 % turbulence): the
    bulk launch takes x-adjacent cell pairs, so the inlet, the outlet and the
    plane that feeds the outlet fall inside the pair rows."""
    from workloads.configs import Workload, _single
    wl = Workload("x96", 96, 48, 48, flow_axis=0, turbulence=0.05,
                  rotors=_single(96, 48, 48, 12.0, 6.0, axis=0))
    rows, eF = _parity_run(P, wl, (1, 50, 150))
    print("t, rel L2 rho, rel L2 u:", rows, "forces", eF)
    for t, e_rho, e_u in rows:
        assert e_rho <= 1e-5 and e_u <= 1e-5, (t, e_rho, e_u)
    assert eF <= 1e-3


def _two_rotors():
    from workloads.configs import RotorSpec, Workload
    return Workload("two48", 48, 48, 128, turbulence=0.05,
                    rotors=[RotorSpec(center=(23.5, 23.5, 32.0), radius=10.0, tsr=6.0),
                            RotorSpec(center=(24.0, 23.0, 88.0), radius=10.0, tsr=5.0, phase0=0.7, pitch=0.05)])


def test_two_rotors_parity(P):
    """Two rotors in tandem (different tip-speed ratio, phase and pitch; the
    second in the first's wake): one embedding, wall-model and force launch
    covers both (one grid row per rotor), each with its own box, lists and
    FP64 sums."""
    wl = _two_rotors()
    rows, eF = _parity_run(P, wl, (1, 40, 120))
    print("two rotors: t, rel L2 rho, rel L2 u:", rows, "forces", eF)
    for t, e_rho, e_u in rows:
        assert e_rho <= 1e-5 and e_u <= 1e-5, (t, e_rho, e_u)
    assert eF <= 1e-3


def test_odd_nx_runs_the_one_cell_kernel(P):
    """nx odd (47x48x96): cell pairs would be misaligned, so the bulk launch
    keeps one cell per thread; fields and forces against the oracle."""
    from workloads.configs import Workload, _single
    wl = Workload("odd47", 47, 48, 96, rotors=_single(47, 48, 96, 12.0, 6.0))
    rows, eF = _parity_run(P, wl, (1, 50, 150))
    print("t, rel L2 rho, rel L2 u:", rows, "forces", eF)
    for t, e_rho, e_u in rows:
        assert e_rho <= 1e-5 and e_u <= 1e-5, (t, e_rho, e_u)
    assert eF <= 1e-3


def test_caller_inflow_plane_matches_synthetic_inflow(P):
    """Inlet velocities supplied by the caller each step (the host evaluation
    of the synthetic inflow, copied into the plane between steps) reproduce
    the oracle's run with the Fourier modes; a lattice without an inlet
    refuses a caller plane."""
    import torch
    from workloads.configs import Workload, _single
    from workloads.turbulence import inflow_plane
    wl = Workload("turb48", 48, 48, 96, turbulence=0.05, rotors=_single(48, 48, 96, 12.0, 6.0))
    lat = P.Lattice.from_workload(wl)
    o = O.from_workload(wl)
    plane = torch.empty(lat.inflow_plane_shape(), dtype=torch.float32, device=lat.device)
    lat.set_inflow_plane(plane)
    modes = wl.modes()
    for t in range(120):
        host = torch.from_numpy(inflow_plane(modes, wl.shape, wl.flow_axis, wl.u_in, t).astype(np.float32))
        with torch.cuda.stream(lat.stream):
            plane.copy_(host.pin_memory(), non_blocking=True)
        lat.step(1)
    o.step(120)
    rg, ug = (a.cpu().numpy().astype(np.float64) for a in lat.fields())
    ro, uo = o.fields()
    e_u = _rel_l2(ug[:, 1:-1], uo[:, 1:-1])
    e_rho = float(np.linalg.norm((rg - ro)[1:-1]) / np.linalg.norm(ro[1:-1]))
    print("caller plane vs oracle modes, 120 steps: rel L2 rho, u", e_rho, e_u)
    assert e_rho <= 1e-5 and e_u <= 1e-5
    lat.set_inflow_plane(None)
    closed = P.Lattice(16, 16, 16, open_boundaries=False)
    with pytest.raises(P.HlError):
        closed.set_inflow_plane(torch.zeros(closed.inflow_plane_shape(), device=closed.device))


def test_loads_async_matches_forces_and_moments(P):
    """hl_loads_async copies each step's force and torque into pinned host
    memory without synchronising; read after an event, they equal what
    hl_forces and hl_moments report for the same step."""
    import torch
    wl = _wl48()
    lat = P.Lattice.from_workload(wl)
    ring = torch.zeros((3, 1, 6), dtype=torch.float64).pin_memory()
    evs = [torch.cuda.Event() for _ in range(3)]
    ref = []
    for i in range(3):
        lat.step_async(1)
        lat.loads_async(ring[i])
        evs[i].record(lat.stream)
        lat.check()
        F, _ = lat.forces()
        M, _ = lat.moments()
        ref.append(np.concatenate([F[0], M[0]]))
    for i in range(3):
        evs[i].synchronize()
        assert np.array_equal(ring[i, 0].numpy(), ref[i]), (i, ring[i, 0].numpy(), ref[i])
    assert not np.array_equal(ref[0], ref[2])
