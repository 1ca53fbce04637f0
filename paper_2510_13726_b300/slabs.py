"""Domain decomposition of a lattice along z into slabs.

The paper scales its wall-modelled rotor runs out by domain decomposition
with one rotor per GPU (Sec. 5, weak scaling of the wind farm): every GPU
advances its own block of cells, neighbouring blocks exchange the
populations that cross their common face each step, and the loads of each
rotor are reduced.  Here the blocks are slabs of whole z planes (z is the
slowest axis in memory, so a face is one contiguous plane per slot):

* each slab is a ``Lattice`` with halo planes on the faces it shares with
  another slab (``halo_lo`` / ``halo_hi`` of the C ABI); with the flow along
  z the first slab keeps the inlet and the last the outlet;
* in the AA pattern only odd steps move populations between cells, so every
  odd step is bracketed by exchanges (one after the even step before it, one
  after it): each shared face sends one message (one plane of the 5 or 9
  slots whose velocity crosses the face) each way, ``hl_halo_export`` on one
  side and ``hl_halo_import`` on the other;
* a face may cut a rotor's box: both slabs then keep ``deep`` halo planes
  there (enough for the wall-model sample to reach through the face), and
  after the one-plane exchange every such face also moves every slot of
  those planes (``hl_halo_deep_export`` / ``hl_halo_deep_import``), before
  the first step too.  Each slab embeds, models and collides the part of the
  box in its own planes; the rotor's force and torque are the sum of the
  slabs' shares;
* a transport carries the messages: a device copy when both slabs live in
  this process, point-to-point messages of ``torch.distributed`` (NCCL on
  GPUs) between ranks;
* the loads are reduced over the ranks as ``[n_rotors][12]`` doubles (F, M
  and their running means).

Every step of the path runs in the library's kernels; this module only
orders calls and moves buffers.
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np


# halo planes of a face that cuts a rotor box: the wall-model sample (y_s = 2
# cells along the normal, trilinear corners) and the plane its odd-step
# corner velocities are gathered from (the library's rule, ceil(y_s) + 2)
def deep_halo(wm_ysample: float = 2.0) -> int:
    return int(math.ceil(wm_ysample)) + 2


@dataclasses.dataclass
class SlabSpec:
    """Slab k of K: global planes z_lo <= z < z_hi, and the halo planes of its
    lower and upper face (0: no shared face; 1: a plain shared face; more: a
    face that cuts a rotor box)."""
    k: int
    z_lo: int
    z_hi: int
    halo_lo: int
    halo_hi: int

    @property
    def z_offset(self) -> int:
        """Global z of the slab's local plane 0."""
        return self.z_lo - int(self.halo_lo)

    @property
    def nz_local(self) -> int:
        return self.z_hi - self.z_lo + int(self.halo_lo) + int(self.halo_hi)


def rotor_z_extent(grid, center, axis, eps_h=2.0):
    """Planes [a, b] of a rotor's box along z: every cell the blades or the
    hub can reach at any angle and pitch, plus two cells (the rule the
    library applies when the rotor is set; it rejects a box that does not
    fit the slab)."""
    h = grid.spacing
    gz, gy, gx = grid.sdf.shape
    rmax = max(abs(grid.origin[0]), abs(grid.origin[0] + h * (gx - 1)))
    tmax = max(abs(grid.origin[1]), abs(grid.origin[1] + h * (gy - 1)))
    amax = max(abs(grid.origin[2]), abs(grid.origin[2] + h * (gz - 1)))
    w = math.hypot(tmax, amax)
    hub = grid.hub_radius + 0.5 * eps_h if grid.hub_radius > 0 else 0.0
    reach = max(w, hub) if axis == 2 else max(math.hypot(rmax, w), hub)
    reach += 2.0
    return int(math.floor(center[2] - reach)), int(math.ceil(center[2] + reach))


def partition(nz: int, parts: int, extents=(), split_boxes: bool = False) -> list:
    """Cut planes [0, c_1, ..., nz] of `parts` slabs of nearly equal depth.
    Unless `split_boxes`, each cut is moved off any rotor box it would split
    (to the nearer box edge; ValueError if no such cut exists)."""
    if parts < 1 or parts > nz:
        raise ValueError("need 1 <= parts <= nz")
    cuts = [0]
    for k in range(1, parts):
        c = int(round(k * nz / parts))
        if not split_boxes:
            for a, b in extents:
                if a < c <= b:
                    c = a if c - a <= b + 1 - c else b + 1
        if not cuts[-1] < c < nz:
            raise ValueError(f"no cut between rotor boxes near plane {round(k * nz / parts)}")
        if not split_boxes:
            for a, b in extents:
                if a < c <= b:
                    raise ValueError(f"cut {c} splits a rotor box [{a}, {b}]")
        cuts.append(c)
    cuts.append(nz)
    return cuts


def cuts_in_boxes(cuts, extents, nz: int, periodic_z: bool) -> set:
    """Indices k of the cut planes cuts[k] (the face below slab k; with z
    periodic cut 0 is also the face above the last slab) that fall inside a
    rotor box [a, b], i.e. a < cuts[k] <= b."""
    out = set()
    for k, c in enumerate(cuts[:-1]):
        if k == 0 and not periodic_z:
            continue
        for a, b in extents:
            if a < c <= b or (k == 0 and (a < c + nz <= b or a < c - nz <= b)):
                out.add(k)
    return out


def slab_specs(cuts, periodic_z: bool, deep=(), depth: int = 4) -> list:
    """Slabs of a cut list.  Shared faces get one halo plane, or `depth`
    where the cut's index is in `deep` (it cuts a rotor box); with z periodic
    the first and last slab share a face (a single periodic slab needs
    none)."""
    K = len(cuts) - 1
    out = []
    for k in range(K):
        lo_shared = k > 0 or (periodic_z and K > 1)
        hi_shared = k < K - 1 or (periodic_z and K > 1)
        lo = (depth if k in deep else 1) if lo_shared else 0
        hi = (depth if ((k + 1) % K) in deep else 1) if hi_shared else 0
        out.append(SlabSpec(k, cuts[k], cuts[k + 1], lo, hi))
    return out


class SlabDomain:
    """A lattice decomposed along z; this process holds the slabs `held`.

    ``engines[k]`` is the ``Lattice`` (or any object with the same halo and
    step calls) of held slab k; ``rank_of[k]`` the rank that holds slab k
    (all this rank's when None); ``group`` the torch.distributed group for
    messages between ranks and the load reduction; ``rotor_slab[r]`` the
    (slab, local rotor id) pairs that hold a share of global rotor r."""

    def __init__(self, specs, engines: dict, rank_of=None, group=None, rotor_slab=None):
        self.specs = list(specs)
        self.K = len(self.specs)
        self.engines = dict(engines)
        self.held = sorted(self.engines)
        self.rank_of = list(rank_of) if rank_of is not None else [None] * self.K
        self.group = group
        self.rotor_slab = [list(v) if isinstance(v, list) else [tuple(v)] for v in (rotor_slab or [])]
        self._bufs = {}
        for k in self.held:
            for f in self._faces(k):
                self._bufs[(k, f, "in")] = self._alloc(k, self.engines[k].halo_size())
                self._bufs[(k, f, "out")] = self._alloc(k, self.engines[k].halo_size())
                if self._deep(k, f):
                    n = self.engines[k].halo_deep_size(f)
                    self._bufs[(k, f, "deep_in")] = self._alloc(k, n)
                    self._bufs[(k, f, "deep_out")] = self._alloc(k, n)
        self._deep_t = None     # time of the last deep exchange

    # -- topology -----------------------------------------------------------
    def _faces(self, k):
        s = self.specs[k]
        return [f for f, on in ((0, s.halo_lo), (1, s.halo_hi)) if on]

    def _deep(self, k, f):
        """Face f of slab k cuts a rotor box (more than one halo plane)."""
        s = self.specs[k]
        return (s.halo_lo if f == 0 else s.halo_hi) > 1

    def _neighbour(self, k, face):
        return (k - 1) % self.K if face == 0 else (k + 1) % self.K

    def _alloc(self, k, nbytes):
        import torch
        e = self.engines[k]
        return torch.empty(nbytes, dtype=torch.uint8, device=getattr(e, "device", "cpu"))

    @property
    def t(self) -> int:
        return self.engines[self.held[0]].t

    # -- time loop ----------------------------------------------------------
    def _move(self, kind, faces):
        """Carry the `kind` messages of `faces` ((slab, face) pairs of held
        slabs) to the neighbours: a copy within the process, else one
        point-to-point message per (sender slab, sender face), posted by both
        sides in the order of that key so that pairs match."""
        sends, recvs = [], []
        for k, f in faces:
            nb, nf = self._neighbour(k, f), 1 - f
            if nb in self.engines:
                self._bufs[(k, f, kind + "in")].copy_(self._bufs[(nb, nf, kind + "out")])
            else:
                sends.append(((k, f), self.rank_of[nb], self._bufs[(k, f, kind + "out")]))
                recvs.append(((nb, nf), self.rank_of[nb], self._bufs[(k, f, kind + "in")]))
        if sends or recvs:
            import torch.distributed as dist
            base = 0 if kind == "" else 2 * self.K
            ops = [dist.P2POp(dist.isend, buf, peer, group=self.group, tag=base + 2 * key[0] + key[1])
                   for key, peer, buf in sorted(sends, key=lambda m: m[0])]
            ops += [dist.P2POp(dist.irecv, buf, peer, group=self.group, tag=base + 2 * key[0] + key[1])
                    for key, peer, buf in sorted(recvs, key=lambda m: m[0])]
            for req in dist.batch_isend_irecv(ops):
                req.wait()

    def _deep_exchange(self):
        faces = [(k, f) for k in self.held for f in self._faces(k) if self._deep(k, f)]
        if not faces:
            return
        for k, f in faces:
            self.engines[k].halo_deep_export(f, self._bufs[(k, f, "deep_out")])
        self._move("deep_", faces)
        for k, f in faces:
            self.engines[k].halo_deep_import(f, self._bufs[(k, f, "deep_in")])
        self._deep_t = self.t

    def exchange(self):
        """Move every halo message once (both directions of every shared face);
        then, on faces that cut a rotor box, the deep messages (every slot of
        the planes next to the face), which need the neighbours' boundary
        planes complete."""
        faces = [(k, f) for k in self.held for f in self._faces(k)]
        for k, f in faces:
            self.engines[k].halo_export(f, self._bufs[(k, f, "out")])
        self._move("", faces)
        for k, f in faces:
            self.engines[k].halo_import(f, self._bufs[(k, f, "in")])
        self._deep_exchange()

    def step(self, n: int = 1):
        """Advance every slab n steps, with one exchange after every step: after
        an even step it fills the halos the odd step reads, after an odd step it
        returns what the odd step wrote there.  Between steps every slab is
        then complete (fields and checkpoints need no further exchange).  Deep
        halos are filled before the first step too."""
        if int(n) > 0 and self._deep_t != self.t:
            self._deep_exchange()
        for _ in range(int(n)):
            for k in self.held:
                self.engines[k].step_async(1)
            self.exchange()
        for k in self.held:
            self.engines[k].check()

    # -- results ------------------------------------------------------------
    def _reduce(self, arr: np.ndarray) -> np.ndarray:
        if self.group is None and all(r is None for r in self.rank_of):
            return arr
        import torch
        import torch.distributed as dist
        t = torch.tensor(arr, dtype=torch.float64)
        if dist.get_backend(self.group) == "nccl":
            t = t.cuda()
        dist.all_reduce(t, group=self.group)
        return t.cpu().numpy()

    def loads(self):
        """(F, F_avg, M, M_avg) of every rotor, each (n_rotors, 3): the sum of
        the shares of the slabs that hold part of its box, reduced over the
        ranks."""
        nrot = len(self.rotor_slab)
        acc = np.zeros((max(nrot, 1), 12))
        for r, parts in enumerate(self.rotor_slab):
            for k, rid in parts:
                if k in self.engines:
                    e = self.engines[k]
                    F, Fa = e.forces()
                    M, Ma = e.moments()
                    acc[r] += np.concatenate([F[rid], Fa[rid], M[rid], Ma[rid]])
        acc = self._reduce(acc)[:nrot]
        return acc[:, 0:3], acc[:, 3:6], acc[:, 6:9], acc[:, 9:12]

    def mass(self) -> float:
        """FP64 total mass of the owned cells of every slab."""
        m = np.array([sum(self.engines[k].mass() for k in self.held)])
        return float(self._reduce(m)[0])

    def fields(self):
        """(rho (nz, ny, nx), u (3, nz, ny, nx)) of the whole lattice as device
        tensors; every slab must be held by this process."""
        import torch
        if len(self.held) != self.K:
            raise RuntimeError("fields() gathers the whole lattice: hold every slab")
        rs, us = [], []
        for k in self.held:
            s = self.specs[k]
            rho, u = self.engines[k].fields()
            a = int(s.halo_lo)
            b = a + (s.z_hi - s.z_lo)
            rs.append(rho[a:b])
            us.append(u[:, a:b])
        return torch.cat(rs, 0), torch.cat(us, 1)

    def close(self):
        for e in self.engines.values():
            if hasattr(e, "close"):
                e.close()
        self.engines = {}

    # -- construction ---------------------------------------------------------
    @classmethod
    def from_workload(cls, wl, parts=None, cuts=None, held=None, rank_of=None, group=None, storage="f32",
                      split_boxes=False, **overrides):
        """Slabs of a ``workloads.Workload`` (rotor axes and centres global).
        `cuts` (global cut planes) or `parts` (number of slabs; cuts placed
        between rotor boxes unless `split_boxes`); a cut inside a rotor box
        gets deep halo planes on both sides and the rotor a share in every slab
        its box reaches.  `held`: the slabs this process builds (all by
        default)."""
        from .lattice import Lattice
        grids = wl.blade_grids()
        ext = [rotor_z_extent(g, r.center, wl.flow_axis, wl.eps_h) for r, g in zip(wl.rotors, grids)]
        if cuts is None:
            cuts = partition(wl.nz, parts or 1, ext, split_boxes=split_boxes)
        periodic_z = not (overrides.get("open_boundaries", True) and wl.flow_axis == 2)
        for a, b in ext:
            if periodic_z and (a < 0 or b >= wl.nz):
                raise ValueError(f"rotor box [{a}, {b}] crosses the periodic z face")
        deep = cuts_in_boxes(cuts, ext, wl.nz, periodic_z)
        specs = slab_specs(cuts, periodic_z, deep, deep_halo(overrides.get("wm_ysample", 2.0)))
        held = list(range(len(specs))) if held is None else list(held)
        kw = dict(q=wl.q, storage=storage, flow_axis=wl.flow_axis, tau_mo=wl.tau_mo, c_smag=wl.c_smag,
                  u_in=wl.u_in, eps_h=wl.eps_h, modes=wl.modes())
        kw.update(overrides)
        engines, rotor_slab = {}, []
        for k in held:
            s = specs[k]
            engines[k] = Lattice(wl.nx, wl.ny, s.nz_local, halo_lo=s.halo_lo, halo_hi=s.halo_hi,
                                 z_offset=s.z_offset, **kw)
        counts = [0] * len(specs)
        for spec, g, (a, b) in zip(wl.rotors, grids, ext):
            parts_r = []
            for s in specs:
                if a >= s.z_hi or b < s.z_lo:
                    continue                       # the box misses the slab's planes
                rid = counts[s.k]
                counts[s.k] += 1
                parts_r.append((s.k, rid))
                if s.k in engines:
                    c = list(spec.center)
                    c[2] -= s.z_offset
                    engines[s.k].add_rotor(g, center=tuple(c), omega=spec.omega(wl.u_in), pitch=spec.pitch,
                                           phase0=spec.phase0, n_blades=spec.n_blades)
            rotor_slab.append(parts_r)
        return cls(specs, engines, rank_of=rank_of, group=group, rotor_slab=rotor_slab)
