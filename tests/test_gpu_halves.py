"""AA layout with x halves (layout 2): each x row of a population slot holds
its two halves interleaved, and the bulk launch takes the cell pairs
(x, x + nx/2), one aligned access per slot at both step parities.  The cell
model is the same; which cells take the packed path and which the per-cell
path differs between the layouts (the x-halves launch also packs the rows on
periodic y and z faces at odd steps), so the two agree to the rounding of
the two paths.  The parity of this layout with the FP64 oracle is in
test_gpu_rotor128.py; slabs in this layout equal the whole lattice bit for
bit; the gradient sweep runs on the AA form of the state.
"""

import numpy as np
import pytest

from workloads.configs import Workload, _single

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("a CUDA device is required for the gpu-marked tests")
    from paper_2510_13726_b300.build import build
    build()
    import paper_2510_13726_b300 as P
    return P


def _random_fields(shape, seed):
    import torch
    nz, ny, nx = shape
    g = np.random.default_rng(seed)
    rho = 1.0 + 0.01 * g.standard_normal(nz * ny * nx)
    u = 0.03 * g.standard_normal((3, nz * ny * nx))
    return torch.tensor(rho, dtype=torch.float32), torch.tensor(u, dtype=torch.float32)


def _pair(P, nx, ny, nz, **kw):
    a = P.Lattice(nx, ny, nz, layout="aa", **kw)
    b = P.Lattice(nx, ny, nz, layout="aa_halves", **kw)
    return a, b


def _rel(a, b):
    a = a.double()
    b = b.double()
    return float((a - b).norm() / a.norm())


@pytest.mark.parametrize("q,storage", [(19, "f32"), (19, "f16s"), (19, "bf16s"), (27, "f32"), (27, "bf16s")])
def test_periodic_lattice_agrees_with_aa(P, q, storage):
    """Periodic 64x20x12 lattice from a random field, 30 steps.  Every pair
    takes the packed path in the x-halves layout, also on the periodic y and z
    faces at odd steps (with wrapped row offsets), where the AA layout falls
    back to the per-cell path: the two agree to the rounding of the two paths
    (FP32: relative L2 of u within 1e-6 and of rho - 1 (about 1e-2, so FP32
    rounding of rho near 1 weighs 1e2 times more) within 1e-5; 16-bit storage
    carries a differently rounded value on to the next step at the storage
    precision: 2e-3 for FP16, 2e-2 for BF16 with its 8 significant bits).
    A wrong row or slot offset would show at order one."""
    nx, ny, nz = 64, 20, 12
    a, b = _pair(P, nx, ny, nz, q=q, storage=storage, open_boundaries=False, wall_model=False)
    rho, u = _random_fields((nz, ny, nx), 3)
    a.init_fields(rho, u)
    b.init_fields(rho, u)
    tol_rho, tol_u = {"f32": (1e-5, 1e-6), "f16s": (2e-3, 2e-3), "bf16s": (2e-2, 2e-2)}[storage]
    for t in (1, 2, 7, 30):
        a.step(t - a.t)
        b.step(t - b.t)
        ra, ua = a.fields()
        rb, ub = b.fields()
        e = (_rel(ra - 1.0, rb - 1.0), _rel(ua, ub))
        assert e[0] <= tol_rho and e[1] <= tol_u, (q, storage, t, e)
    # mass: FP32 collisions conserve it to rounding on both paths; 16-bit
    # storage rounds every stored value each step
    assert abs(a.mass() - b.mass()) <= {"f32": 1e-9, "f16s": 1e-5, "bf16s": 1e-4}[storage] * abs(a.mass())
    a.close()
    b.close()


@pytest.mark.parametrize("case", ["open_z", "open_y", "open_x", "rotor"])
def test_open_faces_and_rotor_agree_with_aa(P, case):
    """Turbulent inflow through open faces across z, y or x, and a rotor
    (R = 8, wall model on), FP32: other cells take the per-cell path than in
    the AA layout (the pairs (x, x + nx/2) meet the box and the x faces
    elsewhere; the periodic faces take the packed path), so the two agree to
    rounding: relative L2 of u within 1e-6 after 60 steps (1e-5 with the
    rotor, whose wall-function iterations can end one step apart), loads
    within 1e-4; open planes excluded (the scheme leaves them undefined)."""
    axis = {"open_z": 2, "open_y": 1, "open_x": 0, "rotor": 2}[case]
    if case == "rotor":
        wl = Workload("halves_rotor", 64, 48, 64, flow_axis=2, turbulence=0.05, n_modes=16,
                      rotors=_single(64, 48, 64, 8.0, 6.0, axis=2))
    else:
        wl = Workload("halves_open", 64, 24, 32, flow_axis=axis, turbulence=0.05, n_modes=16)
    a = P.Lattice.from_workload(wl, storage="f32", layout="aa")
    b = P.Lattice.from_workload(wl, storage="f32", layout="aa_halves")
    a.step(60)
    b.step(60)
    sl = [slice(None)] * 3
    sl[2 - wl.flow_axis] = slice(1, -1)
    sl = (slice(None),) + tuple(sl)
    err = _rel(a.fields()[1][sl], b.fields()[1][sl])
    print(case, "relative L2 of u between the layouts:", err)
    assert err <= (1e-5 if wl.rotors else 1e-6)
    if wl.rotors:
        Fa, _ = a.forces()
        Fb, _ = b.forces()
        assert np.abs(Fa - Fb).max() <= 1e-4 * np.abs(Fa).max()
    a.close()
    b.close()


def test_slabs_with_x_halves_equal_the_lattice(P):
    """Two slabs in the x-halves layout (BF16) against the whole lattice in
    the same layout, bit for bit on the interior planes."""
    import torch
    from paper_2510_13726_b300.slabs import SlabDomain, rotor_z_extent
    wl = Workload("halves_slabs", 64, 48, 96, flow_axis=2, turbulence=0.05, n_modes=16,
                  rotors=_single(64, 48, 96, 8.0, 6.0, axis=2))
    g = wl.blade_grids()[0]
    _, b = rotor_z_extent(g, wl.rotors[0].center, 2, wl.eps_h)
    whole = P.Lattice.from_workload(wl, storage="bf16s", layout="aa_halves")
    dom = SlabDomain.from_workload(wl, cuts=[0, b + 1, 96], storage="bf16s", layout="aa_halves")
    for t in (1, 2, 7, 40):
        whole.step(t - whole.t)
        dom.step(t - dom.t)
        rw, uw = whole.fields()
        rs, us = dom.fields()
        assert torch.equal(rs[1:-1], rw[1:-1]) and torch.equal(us[:, 1:-1], uw[:, 1:-1]), t
    whole.close()
    dom.close()


@pytest.mark.parametrize("storage,q", [("f32", 19), ("bf16s", 19), ("f32", 27)])
def test_gradient_in_x_halves_equals_aa(P, storage, q):
    """hl_grad on a lattice with x halves permutes the state into the AA
    layout of the same step for the sweep and back: from the same initial
    state the objective equals the AA lattice's to 1e-12, the gradients to the
    rounding of the reverse pass's atomic sums (1e-6), the fields after the
    sweep bit for bit, and after three more steps in each layout to 1e-6."""
    import torch
    wl = Workload("halves_grad", 48, 48, 96, q=q, turbulence=0.05, rotors=_single(48, 48, 96, 12.0, 6.0))
    out = []
    for layout in ("aa", "aa_halves"):
        lat = P.Lattice.from_workload(wl, layout=layout, storage=storage)
        J, gp, gd = lat.grad(11, 5, [1.0], [0.3], ckpt_every=4)
        u_after = lat.fields()[1][:, 1:-1].clone()
        lat.step(3)
        u_more = lat.fields()[1][:, 1:-1].clone()
        out.append((J, float(gp[0]), gd.double().cpu().numpy(), u_after, u_more, lat.t))
        lat.close()
    (Ja, ga, da, ua, va, ta), (Jh, gh, dh, uh, vh, th) = out
    assert th == ta == 14
    assert abs(Jh - Ja) <= 1e-12 * abs(Ja)
    assert abs(gh - ga) <= 1e-6 * abs(ga)
    assert float(np.linalg.norm(dh - da) / np.linalg.norm(da)) <= 1e-6
    assert torch.equal(uh, ua)
    assert _rel(vh, va) <= (1e-6 if storage == "f32" else 2e-3)
