"""Parameter sets of the synthetic rotor workloads.

Each workload is a channel with uniform (optionally turbulent) inflow along
its longest axis, equilibrium inlet/outlet planes on that axis, periodic
lateral boundaries, and one or more three-bladed rotors turning about the
flow axis.  The rotor centre sits on the cross-section centre, one quarter
of the length downstream of the inlet (single-rotor cases).  Lattice units:
spacing 1, time step 1, inflow speed 0.05 (the paper's lattice velocity,
Sec. 4).  Angular velocity = tip-speed ratio * inflow speed / radius.
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np

from .rotor import make_blade_grid
from .turbulence import fourier_modes


@dataclasses.dataclass
class RotorSpec:
    center: tuple
    radius: float
    tsr: float
    phase0: float = 0.0
    pitch: float = 0.0
    n_blades: int = 3

    def omega(self, u_in: float) -> float:
        return self.tsr * u_in / self.radius


@dataclasses.dataclass
class Workload:
    name: str
    nx: int
    ny: int
    nz: int
    q: int = 19
    flow_axis: int = 2
    tau_mo: float = 0.5005
    c_smag: float = 0.1
    u_in: float = 0.05
    eps_h: float = 2.0
    steps: int = 200
    seed: int = 0
    turbulence: float = 0.0          # inflow intensity (0: uniform inflow)
    n_modes: int = 64
    rotors: list = dataclasses.field(default_factory=list)
    note: str = ""
    grid_margin: float = 4.0         # blade-grid padding around the blade (cells)

    @property
    def cells(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def shape(self):
        return (self.nx, self.ny, self.nz)

    def blade_grids(self) -> list:
        """One blade grid per rotor (rotors of equal radius share one grid)."""
        cache = {}
        out = []
        for r in self.rotors:
            if r.radius not in cache:
                cache[r.radius] = make_blade_grid(radius=r.radius, margin=self.grid_margin)
            out.append(cache[r.radius])
        return out

    def modes(self):
        if self.turbulence <= 0.0:
            return None
        length = float(self.shape[self.flow_axis])
        return fourier_modes(self.seed, self.n_modes, length, self.u_in, self.turbulence)


def _single(nx, ny, nz, radius, tsr, axis=2, phase0=0.0, pitch=0.0) -> list:
    n = (nx, ny, nz)
    c = [0.5 * (n[i] - 1) for i in range(3)]
    c[axis] = float(n[axis] // 4)
    return [RotorSpec(center=tuple(c), radius=radius, tsr=tsr, phase0=phase0, pitch=pitch)]


# Gradient workloads take a generic rotor angle and pitch.  At pitch 0 the
# axial blade-frame coordinate of every cell is an integer (the rotor
# centre sits on an integer axial position) and the blade grid has nodes
# every half cell, so every sample lies on a node plane of the grid, where
# the trilinear signed distance has a kink in the pitch direction and the
# pitch derivative is one-sided; the same holds at phase 0 for the first
# blade's in-plane coordinates.
GRADIENT_PHASE0 = 0.37
GRADIENT_PITCH = 0.03


def _farm(seed: int) -> list:
    # 3 rows along x (5 diameters apart, first row one diameter from the
    # inlet) x 2 columns along z; independent seeded phase offsets.
    rng = np.random.Generator(np.random.PCG64(seed + 1000))
    R = 64.0
    D = 2 * R
    rot = []
    for row in range(3):
        for col in range(2):
            c = (D + 5 * D * row, 0.5 * (512 - 1), 255.5 + 512.0 * col)
            rot.append(RotorSpec(center=c, radius=R, tsr=6.0,
                                 phase0=float(2 * math.pi * rng.uniform())))
    return rot


def _make() -> dict:
    w = {}
    w["rotor48"] = Workload(
        "rotor48", 48, 48, 96, steps=200, rotors=_single(48, 48, 96, 12.0, 6.0),
        note="D3Q19, uniform inflow, R=12, TSR 6, 200 steps (oracle size)")
    w["rotor256"] = Workload(
        "rotor256", 256, 256, 512, steps=2000, turbulence=0.05,
        rotors=_single(256, 256, 512, 64.0, 6.0),
        note="D3Q19, 5% turbulent inflow, R=64, TSR 6, 2000 steps")
    w["rotor1024_q27"] = Workload(
        "rotor1024_q27", 512, 512, 1024, q=27, steps=1000,
        rotors=_single(512, 512, 1024, 128.0, 7.0),
        note="D3Q27, R=128, TSR 7, 1000 steps (16-bit storage study)")
    w["rotor256_q27"] = Workload(
        "rotor256_q27", 128, 128, 256, q=27, steps=1000,
        rotors=_single(128, 128, 256, 32.0, 7.0),
        note="D3Q27 128x128x256 sub-run of the 16-bit study, R=32, TSR 7")
    w["rotor128_adj"] = Workload(
        "rotor128_adj", 128, 128, 256, steps=4000,
        rotors=_single(128, 128, 256, 32.0, 6.0, phase0=GRADIENT_PHASE0, pitch=GRADIENT_PITCH),
        note="D3Q19 R=32, 4000 steps, checkpoint every 100 (gradient study)")
    w["rotor48_adj"] = Workload(
        "rotor48_adj", 48, 48, 64, steps=16, rotors=_single(48, 48, 64, 10.0, 6.0, phase0=GRADIENT_PHASE0,
                                                       pitch=GRADIENT_PITCH),
        note="D3Q19 48x48x64, R=10, 16 steps (gradient checks at oracle size)")
    w["farm"] = Workload(
        "farm", 1536, 512, 1024, flow_axis=0, steps=1000, turbulence=0.05,
        rotors=_farm(0),
        note="D3Q19 3x2 rotor array R=64, 5 D streamwise spacing, 1000 steps")
    return w


WORKLOADS = _make()


def workload(name: str) -> Workload:
    return dataclasses.replace(WORKLOADS[name])
