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
* a transport carries the messages: a device copy when both slabs live in
  this process, point-to-point messages of ``torch.distributed`` (NCCL on
  GPUs) between ranks;
* each rotor lives in the slab that contains its whole box (cuts are placed
  between rotor boxes); its force and torque are reduced over the ranks as
  ``[n_rotors][12]`` doubles (F, M and their running means).

Every step of the path runs in the library's kernels; this module only
orders calls and moves buffers.
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class SlabSpec:
    """Slab k of K: global planes z_lo <= z < z_hi, and its halo faces."""
    k: int
    z_lo: int
    z_hi: int
    halo_lo: bool
    halo_hi: bool

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


def partition(nz: int, parts: int, extents=()) -> list:
    """Cut planes [0, c_1, ..., nz] of `parts` slabs of nearly equal depth,
    each cut moved off any rotor box it would split (to the nearer box
    edge).  Raises ValueError if no such cut exists."""
    if parts < 1 or parts > nz:
        raise ValueError("need 1 <= parts <= nz")
    cuts = [0]
    for k in range(1, parts):
        c = int(round(k * nz / parts))
        for a, b in extents:
            if a < c <= b:
                c = a if c - a <= b + 1 - c else b + 1
        if not cuts[-1] < c < nz:
            raise ValueError(f"no cut between rotor boxes near plane {round(k * nz / parts)}")
        for a, b in extents:
            if a < c <= b:
                raise ValueError(f"cut {c} splits a rotor box [{a}, {b}]")
        cuts.append(c)
    cuts.append(nz)
    return cuts


def slab_specs(cuts, periodic_z: bool) -> list:
    """Slabs of a cut list.  Shared faces get halo planes; with z periodic the
    first and last slab share a face (a single periodic slab needs none)."""
    K = len(cuts) - 1
    out = []
    for k in range(K):
        lo_shared = k > 0 or (periodic_z and K > 1)
        hi_shared = k < K - 1 or (periodic_z and K > 1)
        out.append(SlabSpec(k, cuts[k], cuts[k + 1], lo_shared, hi_shared))
    return out


class SlabDomain:
    """A lattice decomposed along z; this process holds the slabs `held`.

    ``engines[k]`` is the ``Lattice`` (or any object with the same halo and
    step calls) of held slab k; ``rank_of[k]`` the rank that holds slab k
    (all this rank's when None); ``group`` the torch.distributed group for
    messages between ranks and the load reduction."""

    def __init__(self, specs, engines: dict, rank_of=None, group=None, rotor_slab=None):
        self.specs = list(specs)
        self.K = len(self.specs)
        self.engines = dict(engines)
        self.held = sorted(self.engines)
        self.rank_of = list(rank_of) if rank_of is not None else [None] * self.K
        self.group = group
        # global rotor r -> (slab, local rotor id)
        self.rotor_slab = list(rotor_slab or [])
        self._bufs = {}
        for k in self.held:
            for f in self._faces(k):
                self._bufs[(k, f, "in")] = self._alloc(k)
                self._bufs[(k, f, "out")] = self._alloc(k)

    # -- topology -----------------------------------------------------------
    def _faces(self, k):
        s = self.specs[k]
        return [f for f, on in ((0, s.halo_lo), (1, s.halo_hi)) if on]

    def _neighbour(self, k, face):
        return (k - 1) % self.K if face == 0 else (k + 1) % self.K

    def _alloc(self, k):
        import torch
        e = self.engines[k]
        return torch.empty(e.halo_size(), dtype=torch.uint8, device=getattr(e, "device", "cpu"))

    @property
    def t(self) -> int:
        return self.engines[self.held[0]].t

    # -- time loop ----------------------------------------------------------
    def exchange(self):
        """Move every halo message once (both directions of every shared face)."""
        for k in self.held:
            for f in self._faces(k):
                self.engines[k].halo_export(f, self._bufs[(k, f, "out")])
        sends, recvs = [], []
        for k in self.held:
            for f in self._faces(k):
                nb, nf = self._neighbour(k, f), 1 - f
                if nb in self.engines:
                    self._bufs[(k, f, "in")].copy_(self._bufs[(nb, nf, "out")])
                else:
                    # one message per (sender slab, sender face): both sides
                    # post in the order of that key, so pairs match in order
                    sends.append(((k, f), self.rank_of[nb], self._bufs[(k, f, "out")]))
                    recvs.append(((nb, nf), self.rank_of[nb], self._bufs[(k, f, "in")]))
        if sends or recvs:
            import torch.distributed as dist
            ops = [dist.P2POp(dist.isend, buf, peer, group=self.group, tag=2 * key[0] + key[1])
                   for key, peer, buf in sorted(sends, key=lambda m: m[0])]
            ops += [dist.P2POp(dist.irecv, buf, peer, group=self.group, tag=2 * key[0] + key[1])
                    for key, peer, buf in sorted(recvs, key=lambda m: m[0])]
            for req in dist.batch_isend_irecv(ops):
                req.wait()
        for k in self.held:
            for f in self._faces(k):
                self.engines[k].halo_import(f, self._bufs[(k, f, "in")])

    def step(self, n: int = 1):
        """Advance every slab n steps, with one exchange after every step: after
        an even step it fills the halos the odd step reads, after an odd step it
        returns what the odd step wrote there.  Between steps every slab is
        then complete (fields and checkpoints need no further exchange)."""
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
        """(F, F_avg, M, M_avg) of every rotor, each (n_rotors, 3), reduced
        over the ranks (a rotor's values come from the slab that holds it)."""
        nrot = len(self.rotor_slab)
        acc = np.zeros((max(nrot, 1), 12))
        for r, (k, rid) in enumerate(self.rotor_slab):
            if k in self.engines:
                e = self.engines[k]
                F, Fa = e.forces()
                M, Ma = e.moments()
                acc[r] = np.concatenate([F[rid], Fa[rid], M[rid], Ma[rid]])
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
                      **overrides):
        """Slabs of a ``workloads.Workload`` (rotor axes and centres global).
        `cuts` (global cut planes) or `parts` (number of slabs, cuts placed
        between rotor boxes); `held`: the slabs this process builds (all by
        default)."""
        from .lattice import Lattice
        grids = wl.blade_grids()
        ext = [rotor_z_extent(g, r.center, wl.flow_axis, wl.eps_h) for r, g in zip(wl.rotors, grids)]
        if cuts is None:
            cuts = partition(wl.nz, parts or 1, ext)
        periodic_z = not (overrides.get("open_boundaries", True) and wl.flow_axis == 2)
        specs = slab_specs(cuts, periodic_z)
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
            k = next((s.k for s in specs if s.z_lo <= a and b < s.z_hi), None)
            if k is None:
                raise ValueError(f"rotor box [{a}, {b}] is split by a cut {cuts}")
            rid = counts[k]
            counts[k] += 1
            rotor_slab.append((k, rid))
            if k in engines:
                c = list(spec.center)
                c[2] -= specs[k].z_offset
                engines[k].add_rotor(g, center=tuple(c), omega=spec.omega(wl.u_in), pitch=spec.pitch,
                                     phase0=spec.phase0, n_blades=spec.n_blades)
        return cls(specs, engines, rank_of=rank_of, group=group, rotor_slab=rotor_slab)
