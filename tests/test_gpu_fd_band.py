"""Hybrid band collision with sigma < 1 on the GPU (Sec. 2.2: the band
cells off the wall set mix the finite-difference Chapman-Enskog term into
their non-equilibrium part) against the FP64 oracle.

* the band-strain kernel's output on the force cells against the oracle's
  central-difference strain of the same pre-collision state;
* whole-step fields and forces of the 48x48x96 rotor with sigma = 0.5
  (D3Q19, wall model on) and sigma = 0 (D3Q27, wall model off);
* the two-stream schedule computes what one stream computes;
* the gradient through the band against the oracle's adjoint;
* the configuration check rejects sigma outside [0, 1].
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


def _rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


@pytest.mark.parametrize("wall_model", [True, False])
def test_band_strain_matches_oracle(P, wall_model):
    wl = W.workload("rotor48")
    lat = P.Lattice.from_workload(wl, sigma_band=0.5, wall_model=wall_model)
    o = O.from_workload(wl, sigma_band=0.5, wall_model=wall_model)
    lat.step(30)
    o.step(30)
    Sref = o.fd_strain()                       # pre-collision state of step 30
    lat.step(1)
    o.step(1)
    band = lat.rotor_band(0)
    lo, n = band["lo"], band["n"]
    fl = band["flags"].cpu().numpy()
    wm = band["wm"].cpu().numpy().astype(np.float64)
    _, _, flo, _ = o.geometry()
    sl = (slice(lo[2], lo[2] + n[2]), slice(lo[1], lo[1] + n[1]), slice(lo[0], lo[0] + n[0]))
    assert np.array_equal(fl & 1, flo[sl] & 1)
    sel = (fl & 1) != 0
    if wall_model:
        sel &= (fl & 2) == 0
    assert sel.sum() > 20
    Sb = Sref[sl][sel]
    ref = np.stack([Sb[:, 0, 0], Sb[:, 1, 1], Sb[:, 2, 2], Sb[:, 0, 1], Sb[:, 0, 2], Sb[:, 1, 2]])
    got = wm[3:9][:, sel]
    scale = np.abs(ref).max()
    err = np.abs(got - ref).max()
    print("band strain cells, max |S|, max error:", int(sel.sum()), scale, err)
    assert scale > 1e-4
    assert err <= 1e-4 * scale, (err, scale)


@pytest.mark.parametrize("q,sigma,wall_model", [(19, 0.5, True), (27, 0.0, False)])
def test_whole_step_parity_hybrid_band(P, q, sigma, wall_model):
    wl = W.workload("rotor48")
    wl.q = q
    lat = P.Lattice.from_workload(wl, sigma_band=sigma, wall_model=wall_model)
    o = O.from_workload(wl, sigma_band=sigma, wall_model=wall_model)
    ref = O.from_workload(wl, wall_model=wall_model)
    report = []
    for t_target in (1, 50, 150):
        lat.step(t_target - lat.t)
        o.step(t_target - o.t)
        ref.step(t_target - ref.t)
        rg, ug = (a.cpu().numpy().astype(np.float64) for a in lat.fields())
        ro, uo = o.fields()
        _, u1 = ref.fields()
        e_rho = np.linalg.norm((rg - ro)[1:-1]) / np.linalg.norm(ro[1:-1])
        e_u = _rel_l2(ug[:, 1:-1], uo[:, 1:-1])
        d_sigma = _rel_l2(uo[:, 1:-1], u1[:, 1:-1])      # how much sigma changes the flow
        report.append((t_target, e_rho, e_u, d_sigma))
    print("t, rel L2 rho, rel L2 u, effect of sigma:", report)
    for t, e_rho, e_u, d_sigma in report:
        assert e_rho <= 1e-5 and e_u <= 1e-5, (t, e_rho, e_u)
    assert report[-1][3] > 20 * report[-1][2]
    Fg, _ = lat.forces()
    Fo, _, _, _ = o.forces()
    assert np.abs(Fg - Fo).max() <= 1e-3 * np.abs(Fo).max()


def test_overlap_schedule_bit_identical_with_hybrid_band(P):
    import torch
    wl = W.workload("rotor48")
    a = P.Lattice.from_workload(wl, sigma_band=0.5, overlap=True)
    b = P.Lattice.from_workload(wl, sigma_band=0.5, overlap=False)
    a.step(23)
    b.step(23)
    assert torch.equal(a.fields()[1], b.fields()[1])
    Fa, _ = a.forces()
    Fb, _ = b.forces()
    assert np.allclose(Fa, Fb, rtol=1e-12, atol=0)


@pytest.mark.parametrize("wall_model,q", [(False, 19), (True, 19), (False, 27)])
def test_gradient_parity_with_oracle(P, wall_model, q):
    """hl_grad with sigma = 0.5 (the box adjoint hands the strain sensitivity
    of the hybrid band cells to adj_band_strain_kernel, which passes it to
    the neighbours' populations) against the oracle's adjoint: J, dJ/dpitch
    and dJ/dd0 of J = mean over the last 8 of 16 steps of thrust - 0.3
    torque, checkpoints every 5 steps; the lattice ends where hl_step leaves
    it."""
    import torch
    wl = W.workload("rotor48_adj")
    wl.q = q
    T, navg, wT, wQ = 16, 8, 1.0, -0.3
    lat = P.Lattice.from_workload(wl, wall_model=wall_model, sigma_band=0.5)
    Jg, gpg, gdg = lat.grad(T, navg, [wT], [wQ], ckpt_every=5)
    gdg = gdg.cpu().numpy().astype(np.float64)
    o = O.from_workload(wl, wall_model=wall_model, sigma_band=0.5)
    Jo, gpo, gdo = o.adjoint(T, navg, [wT], [wQ])
    print(f"J {Jg:.8e} vs {Jo:.8e}; dJ/dpitch {gpg[0]:.8e} vs {gpo[0]:.8e}; "
          f"dJ/dd0 rel L2 {_rel_l2(gdg, gdo):.2e}")
    assert abs(Jg - Jo) <= 1e-5 * abs(Jo)
    assert abs(gpg[0] - gpo[0]) <= 1e-4 * abs(gpo[0])
    assert _rel_l2(gdg, gdo) <= 1e-4
    ref = P.Lattice.from_workload(wl, wall_model=wall_model, sigma_band=0.5)
    ref.step(T)
    r1, u1 = lat.fields()
    r2, u2 = ref.fields()
    assert torch.equal(r1, r2) and torch.equal(u1, u2)


def test_config_checks(P):
    wl = W.workload("rotor48")
    for bad in (-0.1, 1.5, float("nan")):
        with pytest.raises(Exception):
            P.Lattice.from_workload(wl, sigma_band=bad)
