"""Slab decomposition on one GPU: a lattice split along z into 2 or 3 slabs,
exchanging halo messages through hl_halo_export / hl_halo_import, equals the
undecomposed lattice bit for bit (same kernels, same per-cell arithmetic,
only the place where a population is stored differs), with the rotor box next
to a cut or cut by it (deep halos, hl_halo_deep_export / import); flow along
z (inlet in the first slab, outlet in the last) and flow along x with z
periodic (the last slab wraps onto the first).
"""

import dataclasses

import numpy as np
import pytest

import workloads as W
from workloads.configs import Workload, _single, RotorSpec

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


def _compare(P, wl, cuts, steps, storage="f32", layout="aa", **kw):
    import torch
    from paper_2510_13726_b300.slabs import SlabDomain
    whole = P.Lattice.from_workload(wl, storage=storage, layout=layout, **kw)
    dom = SlabDomain.from_workload(wl, cuts=cuts, storage=storage, layout=layout, **kw)
    # with the flow along z the inlet and outlet planes' fields are not defined
    # by the scheme (at odd steps they read across the open face, where a slab
    # and the whole lattice wrap to different planes): compare the others
    sl = slice(1, -1) if wl.flow_axis == 2 else slice(None)
    for t_target in (1, 2, 7, steps):
        whole.step(t_target - whole.t)
        dom.step(t_target - dom.t)
        rw, uw = whole.fields()
        rs, us = dom.fields()
        assert torch.equal(rs[sl], rw[sl]) and torch.equal(us[:, sl], uw[:, sl]), (
            cuts, t_target, float((us - uw)[:, sl].abs().max()))
    Fw, Faw = whole.forces()
    Mw, Maw = whole.moments()
    F, Fa, M, Ma = dom.loads()
    # the per-rotor FP64 sums run over the same cells in another order
    for a, b in ((F, Fw), (Fa, Faw), (M, Mw), (Ma, Maw)):
        assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()
    # the slabs' owned cells carry the whole lattice's mass
    assert abs(dom.mass() - whole.mass()) <= 1e-12 * whole.mass()
    whole.close()
    dom.close()


def _box_z(wl):
    from paper_2510_13726_b300.slabs import rotor_z_extent
    g = wl.blade_grids()[0]
    return rotor_z_extent(g, wl.rotors[0].center, wl.flow_axis, wl.eps_h)


def test_two_and_three_slabs_equal_the_lattice_flow_along_z(P):
    """rotor48 (48x48x96, R = 12, wall model, flow along z): cuts right after
    the rotor box and at 64; 200 steps."""
    wl = W.workload("rotor48")
    a, b = _box_z(wl)
    _compare(P, wl, [0, b + 1, 96], 200)
    _compare(P, wl, [0, b + 1, 64, 96], 200)
    _compare(P, wl, [0, a, b + 1, 96], 40)          # a slab that is exactly the rotor box


def test_rotor_box_cut_by_slab_faces(P):
    """rotor48 with the cuts inside the rotor box (planes 12..36): through the
    rotor plane (24), two cuts 10 planes apart (20, 30), and a cut two planes
    after the box's start (14).  Faces that cut the box keep 4 halo planes,
    refilled with the neighbour's planes after every step; each slab embeds,
    models and collides its part of the box, the wall-model samples of cells
    next to the face read through it, and the rotor's loads are the sum of the
    slabs' shares (FP64 sums in another order: 1e-12).  200 steps, bit for
    bit on the fields."""
    wl = W.workload("rotor48")
    a, b = _box_z(wl)
    assert (a, b) == (12, 36)
    _compare(P, wl, [0, 24, 96], 200)
    _compare(P, wl, [0, 20, 30, 96], 200)
    _compare(P, wl, [0, 14, 96], 60)


@pytest.mark.parametrize("storage,layout", [("bf16s", "aa"), ("f16s", "aa_halves")])
def test_rotor_box_cut_16bit(P, storage, layout):
    """The cut rotor box with 16-bit storage, in the AA layout and with x halves."""
    _compare(P, W.workload("rotor48"), [0, 22, 96], 60, storage=storage, layout=layout)


def test_rotor_box_cut_with_band_strain(P):
    """sigma = 0.5 on the force cells off the wall set: their finite-difference
    strain gathers the six axis neighbours' velocities, across a cut face from
    the deep halo."""
    _compare(P, W.workload("rotor48"), [0, 24, 96], 100, sigma_band=0.5)


@pytest.mark.parametrize("q", [19, 27])
def test_rotor_boxes_cut_with_z_periodic(P, q):
    """Flow along x with z periodic (the farm's lateral direction): two rotors
    whose boxes (planes 2..37 and 42..77) are each cut by a slab face, plus a
    plain face at the periodic wrap; D3Q19 and D3Q27, 60 steps."""
    R = 8.0
    rot = [RotorSpec(center=(24.0, 23.5, 19.5), radius=R, tsr=6.0, phase0=0.3),
           RotorSpec(center=(24.0, 23.5, 59.5), radius=R, tsr=6.0, phase0=1.9)]
    wl = Workload("pair_x_cut", 95, 48, 80, q=q, flow_axis=0, turbulence=0.05, rotors=rot)
    from paper_2510_13726_b300.slabs import rotor_z_extent
    g = wl.blade_grids()[0]
    ext = [rotor_z_extent(g, r.center, 0, wl.eps_h) for r in rot]
    assert ext[0][0] < 20 <= ext[0][1] and ext[1][0] < 60 <= ext[1][1] and ext[0][0] > 0 and ext[1][1] < 80
    _compare(P, wl, [0, 20, 60, 80], 60)


def test_cut_rotor_box_rules(P):
    """A face that cuts a rotor box needs the deep halo (4 planes with y_s =
    2), no torque drive, and the deep import of every step (also before the
    first); its force reduction runs after the exchange."""
    wl = W.workload("rotor48")
    g = wl.blade_grids()[0]
    rot = wl.rotors[0]
    c = (rot.center[0], rot.center[1], rot.center[2])

    def slab(hi, **kw):
        L = P.Lattice(wl.nx, wl.ny, 24 + hi, halo_hi=hi, **kw)
        return L

    L = slab(1)
    with pytest.raises(P.HlError) as e:
        L.add_rotor(g, center=c, omega=rot.omega(wl.u_in))     # box 12..36 leaves through a 1-plane face
    assert e.value.code == -1
    L.close()
    L = slab(4)
    L.add_rotor(g, center=c, omega=rot.omega(wl.u_in))
    lo, n = L.rotor_box(0)
    assert lo[2] == 12 and lo[2] + n[2] == 24                 # cut at the slab's last owned plane
    with pytest.raises(P.HlError) as e:
        L.set_drive(0, 1e6)
    assert e.value.code == -5
    with pytest.raises(P.HlError) as e:
        L.step(1)                                             # no deep import yet, even at t = 0
    assert e.value.code == -5
    import torch
    buf = torch.empty(L.halo_deep_size(1), dtype=torch.uint8, device=L.device)
    assert L.halo_deep_size(1) == 4 * 19 * wl.nx * wl.ny * 4
    L.halo_deep_export(1, buf)
    L.halo_deep_import(1, buf)
    L.step(1)
    L.close()


def test_slabs_with_turbulent_inflow_and_16bit_storage(P):
    """Turbulent inflow (64 modes, 5 %) and BF16 storage through three slabs."""
    wl = dataclasses.replace(W.workload("rotor48"), turbulence=0.05)
    a, b = _box_z(wl)
    _compare(P, wl, [0, 20 if 20 <= a else a, b + 1, 96], 60, storage="bf16s")


def test_slabs_d3q27(P):
    """D3Q27 (nine populations cross each face): three slabs, rotor box next
    to a cut, FP16 storage."""
    wl = dataclasses.replace(W.workload("rotor48"), q=27)
    a, b = _box_z(wl)
    _compare(P, wl, [0, b + 1, 70, 96], 60, storage="f16s")


def test_periodic_slabs_flow_along_x(P):
    """Flow along x with z periodic (two rotors side by side across z, as the
    wind farm's columns): two slabs, each wrapping onto the other.  nx is odd,
    so every cell takes the one-cell path: with nx even the undecomposed
    lattice's periodic wrap planes (z = 0 and nz - 1) leave the packed pair
    path at odd steps, while in the slabs they are interior planes, and the
    two paths round a few sums in another order."""
    R = 8.0
    rot = [RotorSpec(center=(24.0, 23.5, 19.5), radius=R, tsr=6.0, phase0=0.3),
           RotorSpec(center=(24.0, 23.5, 59.5), radius=R, tsr=6.0, phase0=1.9)]
    wl = Workload("pair_x", 95, 48, 80, flow_axis=0, turbulence=0.05, rotors=rot)
    from paper_2510_13726_b300.slabs import rotor_z_extent
    g = wl.blade_grids()[0]
    ext = [rotor_z_extent(g, r.center, 0, wl.eps_h) for r in rot]
    assert ext[0][0] >= 1 and ext[0][1] < 40 <= ext[1][0] - 1 and ext[1][1] <= 78
    _compare(P, wl, [0, 40, 80], 80)


def test_slab_refuses_steps_without_exchange(P):
    """A slab advances one step per call, and only after the halo exchange of
    its parity."""
    wl = W.workload("rotor48")
    L = P.Lattice(wl.nx, wl.ny, 50, halo_hi=True)
    with pytest.raises(P.HlError) as e:
        L.step(2)
    assert e.value.code == -1
    L.step(1)                                   # t = 0: the even step needs no exchange
    with pytest.raises(P.HlError) as e:
        L.step(1)                               # t = 1 (odd): the upper face has not imported
    assert e.value.code == -5 and L.t == 1
    import torch
    buf = torch.empty(L.halo_size(), dtype=torch.uint8, device=L.device)
    assert L.halo_size() == 5 * wl.nx * wl.ny * 4
    L.halo_export(1, buf)
    L.halo_import(1, buf)                       # a wall of its own: reflects its own plane
    L.step(1)
    with pytest.raises(P.HlError) as e:
        L.halo_export(0, buf)                   # the lower face is the inlet, not a halo
    assert e.value.code == -1
    L.close()
