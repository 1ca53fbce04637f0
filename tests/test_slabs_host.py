"""Host logic of the slab decomposition (no GPU): partition, halo topology,
the halo protocol of the AA pattern, and the exchange between ranks over
torch.distributed (gloo, world size 2).

The engine here is a plain numpy lattice in the AA layout whose collision is
an arbitrary local non-linear map (the decomposition must not depend on what
a cell does with its populations), with halo messages built by the rule the
C ABI documents for hl_halo_export / hl_halo_import.  A decomposed run must
equal the undecomposed one bit for bit; the undecomposed engine itself is
checked against two-buffer pull streaming with np.roll.
"""

import itertools
import os
import socket

import numpy as np
import pytest
import torch

from paper_2510_13726_b300.slabs import SlabDomain, cuts_in_boxes, deep_halo, partition, slab_specs

C19 = np.array([c for c in itertools.product((-1, 0, 1), repeat=3) if sum(abs(v) for v in c) <= 2])
OPP = np.array([int(np.nonzero((C19 == -c).all(1))[0][0]) for c in C19])
W19 = np.array([1 / 3 if not c.any() else (1 / 18 if abs(c).sum() == 1 else 1 / 36) for c in C19])


def local_map(f):
    """Any local, non-linear cell update: relaxation towards a first-order
    equilibrium plus a small non-linear term.  f: (q, ...)."""
    rho = f.sum(0)
    j = np.tensordot(C19.T.astype(float), f, axes=(1, 0))
    feq = W19.reshape((-1,) + (1,) * (f.ndim - 1)) * (rho + 3 * np.tensordot(C19.astype(float), j, axes=(1, 0)))
    return f + 0.6 * (feq - f) + 0.01 * np.sin(7 * f)


class AAEngine:
    """AA-pattern lattice (x, y periodic; z periodic unless it has halo
    planes, which are never updated)."""

    def __init__(self, g, halo_lo=0, halo_hi=0):
        self.g = g.copy()                      # (q, nz, ny, nx): slot s of every cell
        self.halo_lo, self.halo_hi = int(halo_lo), int(halo_hi)
        self.t = 0
        self.device = "cpu"

    def _zr(self):
        nz = self.g.shape[1]
        return range(int(self.halo_lo), nz - int(self.halo_hi))

    def step_async(self, n=1):
        for _ in range(n):
            g = self.g
            new = g.copy()
            zs = list(self._zr())
            if self.t % 2 == 0:
                # even: read own slot s, write own slot opp(s)
                post = local_map(g[:, zs])
                for s in range(19):
                    new[OPP[s], zs] = post[s]
            else:
                # odd: read slot opp(s) of x - c_s, write slot s of x + c_s
                nz, ny, nx = g.shape[1:]
                pre = np.empty((19, len(zs), ny, nx))
                for s in range(19):
                    cx, cy, cz = C19[s]
                    src = np.roll(np.roll(g[OPP[s]], cy, axis=1), cx, axis=2)
                    pre[s] = src[[(z - cz) % nz for z in zs]]
                post = local_map(pre)
                for s in range(19):
                    cx, cy, cz = C19[s]
                    dst = np.roll(np.roll(post[s], cy, axis=1), cx, axis=2)
                    for i, z in enumerate(zs):
                        new[s, (z + cz) % nz] = dst[i]
            self.g = new
            self.t += 1

    def check(self):
        pass

    # halo protocol of include/hlbm.h: the halo plane next to each face and
    # the slab's boundary plane (D halo planes on a face)
    def _plane_sign(self, face, import_):
        nz, odd = self.g.shape[1], self.t % 2 == 1
        h_lo, b_lo = self.halo_lo - 1, self.halo_lo
        h_hi, b_hi = nz - self.halo_hi, nz - self.halo_hi - 1
        if not import_:
            if face == 0:
                return (b_lo, +1) if odd else (h_lo, -1)
            return (b_hi, -1) if odd else (h_hi, +1)
        if face == 0:
            return (h_lo, -1) if odd else (b_lo, +1)
        return (h_hi, +1) if odd else (b_hi, -1)

    def _deep_planes(self, face, import_):
        nz = self.g.shape[1]
        D = self.halo_lo if face == 0 else self.halo_hi
        if face == 0:
            return slice(0, D) if import_ else slice(D, 2 * D)
        return slice(nz - D, nz) if import_ else slice(nz - 2 * D, nz - D)

    def halo_deep_size(self, face):
        D = self.halo_lo if face == 0 else self.halo_hi
        return 19 * D * self.g.shape[2] * self.g.shape[3] * 8

    def halo_deep_export(self, face, buf):
        buf.numpy().view(np.float64)[:] = self.g[:, self._deep_planes(face, False)].ravel()

    def halo_deep_import(self, face, buf):
        sl = self._deep_planes(face, True)
        self.g[:, sl] = buf.numpy().view(np.float64).reshape(self.g[:, sl].shape)

    def halo_size(self):
        return 5 * self.g.shape[2] * self.g.shape[3] * 8

    def halo_export(self, face, buf):
        plane, sign = self._plane_sign(face, False)
        slots = np.nonzero(C19[:, 2] == sign)[0]
        buf.numpy().view(np.float64)[:] = self.g[slots, plane].ravel()

    def halo_import(self, face, buf):
        plane, sign = self._plane_sign(face, True)
        slots = np.nonzero(C19[:, 2] == sign)[0]
        self.g[slots, plane] = buf.numpy().view(np.float64).reshape(len(slots), *self.g.shape[2:])

    def mass(self):
        return float(self.g[:, list(self._zr())].sum())

    def forces(self):
        F = np.array([[self.g[1].sum(), self.t, 1.0]])
        return F, 2 * F

    def moments(self):
        M = np.array([[self.g[2].sum(), -self.t, 3.0]])
        return M, 2 * M


def _initial(shape, seed=3):
    rng = np.random.default_rng(seed)
    return W19[:, None, None, None] * (1 + 0.2 * rng.uniform(-1, 1, (19,) + shape))


def _natural(g, t):
    """f_s(x) before step t from the AA layout."""
    if t % 2 == 0:
        return g.copy()
    out = np.empty_like(g)
    for s in range(19):
        cx, cy, cz = C19[s]
        out[s] = np.roll(g[OPP[s]], (cz, cy, cx), axis=(0, 1, 2))
    return out


def test_aa_engine_matches_pull_streaming():
    """The test engine itself: AA layout == collide, then pull-stream
    f_s(x) <- f*_s(x - c_s) with np.roll, over steps of both parities."""
    g0 = _initial((6, 5, 4))
    e = AAEngine(g0)
    f = g0.copy()
    for t in range(7):
        e.step_async(1)
        post = local_map(f)
        f = np.stack([np.roll(post[s], tuple(C19[s][::-1]), axis=(0, 1, 2)) for s in range(19)])
        assert np.allclose(_natural(e.g, e.t), f, rtol=0, atol=1e-15)


def test_partition_avoids_rotor_boxes():
    assert partition(96, 1) == [0, 96]
    assert partition(96, 2) == [0, 48, 96]
    # a cut c separates planes c - 1 and c; it splits a box [a, b] when a < c <= b
    assert partition(96, 2, [(40, 55)]) == [0, 40, 96]          # moved to the nearer edge
    assert partition(96, 2, [(45, 60)]) == [0, 45, 96]
    assert partition(96, 2, [(30, 47)]) == [0, 48, 96]
    assert partition(96, 3, [(20, 30), (60, 70)]) == [0, 32, 60, 96]
    assert partition(300, 3, [(90, 110), (190, 210)]) == [0, 90, 190, 300]
    with pytest.raises(ValueError):
        partition(20, 2, [(0, 19)])              # the box fills the lattice


def test_slab_specs_topology():
    s = slab_specs([0, 10, 30, 40], periodic_z=False)
    assert [(x.halo_lo, x.halo_hi) for x in s] == [(0, 1), (1, 1), (1, 0)]
    assert [x.nz_local for x in s] == [11, 22, 11] and [x.z_offset for x in s] == [0, 9, 29]
    s = slab_specs([0, 10, 40], periodic_z=True)
    assert [(x.halo_lo, x.halo_hi) for x in s] == [(1, 1), (1, 1)]
    assert slab_specs([0, 40], periodic_z=True)[0].halo_lo == 0
    # a cut inside a rotor box gets deep halo planes on both sides
    assert cuts_in_boxes([0, 30, 60, 96], [(20, 40)], 96, False) == {1}
    assert cuts_in_boxes([0, 30, 60, 96], [(30, 40)], 96, False) == set()     # cut at the box's first plane
    assert cuts_in_boxes([0, 48, 96], [(-5, 10)], 96, True) == {0}            # across the periodic face
    s = slab_specs([0, 30, 60, 96], periodic_z=False, deep={1}, depth=4)
    assert [(x.halo_lo, x.halo_hi) for x in s] == [(0, 4), (4, 1), (1, 0)]
    assert [x.nz_local for x in s] == [34, 35, 37] and [x.z_offset for x in s] == [0, 26, 59]
    s = slab_specs([0, 30, 60], periodic_z=True, deep={0}, depth=3)
    assert [(x.halo_lo, x.halo_hi) for x in s] == [(3, 1), (1, 3)]
    assert partition(96, 2, [(40, 55)], split_boxes=True) == [0, 48, 96]
    assert deep_halo(2.0) == 4 and deep_halo(2.5) == 5


def _slab_engines(g0, cuts, held, deep=(), depth=1):
    specs = slab_specs(cuts, periodic_z=True, deep=deep, depth=depth)
    nz = g0.shape[1]
    eng = {}
    for k in held:
        s = specs[k]
        zs = [(z - int(s.halo_lo)) % nz for z in range(s.z_lo, s.z_lo + s.nz_local)]
        eng[k] = AAEngine(g0[:, zs], s.halo_lo, s.halo_hi)
    return specs, eng


def _run_slabs(cuts, held, steps, rank_of=None, group=None, shape=(12, 5, 4), deep=(), depth=1):
    g0 = _initial(shape)
    specs, eng = _slab_engines(g0, cuts, held, deep, depth)
    dom = SlabDomain(specs, eng, rank_of=rank_of, group=group, rotor_slab=[(k, 0) for k in range(len(specs))])
    dom.step(steps)
    return dom, specs


@pytest.mark.parametrize("cuts", [[0, 5, 12], [0, 3, 7, 12], [0, 2, 4, 6, 8, 10, 12]])
def test_local_slabs_equal_the_whole_lattice(cuts):
    """All slabs in one process (device copies): the owned planes equal the
    undecomposed lattice bit for bit after steps of both parities."""
    whole = AAEngine(_initial((12, 5, 4)))
    whole.step_async(9)
    dom, specs = _run_slabs(cuts, range(len(cuts) - 1), 9)
    for s in specs:
        e = dom.engines[s.k]
        a = int(s.halo_lo)
        assert np.array_equal(e.g[:, a:a + s.z_hi - s.z_lo], whole.g[:, s.z_lo:s.z_hi]), s
    assert abs(dom.mass() - whole.g.sum()) < 1e-12 * whole.g.sum()


@pytest.mark.parametrize("cuts,deep,depth", [([0, 6, 12], {1}, 3), ([0, 5, 12], {0, 1}, 4),
                                              ([0, 4, 8, 12], {2}, 2)])
def test_deep_halos_carry_the_neighbours_state(cuts, deep, depth):
    """Faces that cut a rotor box keep D halo planes, refilled after every
    step (after the one-plane exchange) with every slot of the neighbour's
    D planes next to the face, and before the first step.  Between steps:
    the owned planes equal the undecomposed lattice, the deep halo planes
    hold exactly the lattice's planes there (every slot), and the
    pre-collision populations of the halo cells (every plane but the one
    farthest from the face, whose odd-step populations sit one plane
    further) equal the lattice's, at both parities: what the wall-model
    sample and the force reduction read through the face."""
    shape = (12, 5, 4)
    nz = shape[0]
    g0 = _initial(shape)
    whole = AAEngine(g0)
    specs, eng = _slab_engines(g0, cuts, range(len(cuts) - 1), deep, depth)
    dom = SlabDomain(specs, eng)
    for t in range(1, 9):
        dom.step(1)
        whole.step_async(1)
        nat_w = _natural(whole.g, whole.t)
        for sp in specs:
            e = dom.engines[sp.k]
            a = sp.halo_lo
            assert np.array_equal(e.g[:, a:a + sp.z_hi - sp.z_lo], whole.g[:, sp.z_lo:sp.z_hi]), (t, sp)
            nat_s = _natural(e.g, e.t)
            for f, D in ((0, sp.halo_lo), (1, sp.halo_hi)):
                if D < 2:
                    continue
                loc = range(0, D) if f == 0 else range(e.g.shape[1] - D, e.g.shape[1])
                for zl in loc:
                    zg = (zl + sp.z_offset) % nz
                    assert np.array_equal(e.g[:, zl], whole.g[:, zg]), (t, sp, f, zl)
                    farthest = zl == (0 if f == 0 else e.g.shape[1] - 1)
                    if not farthest:
                        assert np.array_equal(nat_s[:, zl], nat_w[:, zg]), (t, sp, f, zl)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, cuts, held_of, steps, out_dir, deep=(), depth=1):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        rank_of = [r for k in range(len(cuts) - 1) for r in range(world) if k in held_of[r]]
        dom, specs = _run_slabs(cuts, held_of[rank], steps, rank_of=rank_of, group=dist.group.WORLD,
                                deep=deep, depth=depth)
        F, Fa, M, Ma = dom.loads()
        res = {"mass": dom.mass(), "F": F, "M": M}
        for k in dom.held:
            res[f"g{k}"] = dom.engines[k].g
        np.savez(os.path.join(out_dir, f"rank{rank}.npz"), **res)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("cuts,held_of,deep,depth", [([0, 6, 12], [[0], [1]], (), 1),
                                                     ([0, 3, 7, 12], [[0, 1], [2]], (), 1),
                                                     ([0, 6, 12], [[0], [1]], {0, 1}, 3),
                                                     ([0, 4, 8, 12], [[0, 2], [1]], {1}, 2)])
def test_slabs_over_two_gloo_ranks(tmp_path, cuts, held_of, deep, depth):
    """Slabs split over two processes (gloo): messages between ranks through
    torch.distributed point-to-point, between slabs of one rank by copies;
    faces that cut a rotor box also move their deep messages (tagged apart
    from the one-plane ones).  Every slab equals the undecomposed lattice bit
    for bit, deep halos included; the mass and the per-rotor loads (one
    'rotor' per slab here) are reduced over the ranks."""
    import torch.multiprocessing as mp
    steps = 9
    mp.spawn(_rank_main, args=(2, _free_port(), cuts, held_of, steps, str(tmp_path), deep, depth), nprocs=2,
             join=True)
    whole = AAEngine(_initial((12, 5, 4)))
    whole.step_async(steps)
    specs = slab_specs(cuts, periodic_z=True, deep=deep, depth=depth)
    got = [dict(np.load(tmp_path / f"rank{r}.npz")) for r in range(2)]
    for r in range(2):
        for k in held_of[r]:
            s = specs[k]
            a = int(s.halo_lo)
            assert np.array_equal(got[r][f"g{k}"][:, a:a + s.z_hi - s.z_lo], whole.g[:, s.z_lo:s.z_hi])
            # deep halo planes hold the neighbours' planes
            for zl in list(range(s.halo_lo if s.halo_lo > 1 else 0)) + \
                    list(range(s.nz_local - (s.halo_hi if s.halo_hi > 1 else 0), s.nz_local)):
                assert np.array_equal(got[r][f"g{k}"][:, zl], whole.g[:, (zl + s.z_offset) % 12])
        assert abs(got[r]["mass"] - whole.g.sum()) < 1e-12 * whole.g.sum()
    assert np.array_equal(got[0]["F"], got[1]["F"]) and np.array_equal(got[0]["M"], got[1]["M"])
    assert got[0]["F"].shape == (len(specs), 3) and np.all(got[0]["F"][:, 1] == steps)
