"""Seeded synthetic inputs shared by the FP64 oracle and the CUDA library.

This package produces *data* only: the voxelised blade signed-distance grid
of a NACA 4412 rotor, the random-Fourier-mode table of the turbulent inflow,
random population states for unit tests, and the parameter sets of the
rotor workloads.  It performs none of the lattice Boltzmann arithmetic
(no moments, equilibria, collisions, porosity, wall model or forces), and it
imports neither ``oracle`` nor ``paper_2510_13726_b300``.
"""

from .rotor import BladeGrid, naca4_polygon, make_blade_grid, blade_box_extent
from .turbulence import fourier_modes
from .states import random_populations
from .configs import Workload, RotorSpec, workload, WORKLOADS

__all__ = [
    "BladeGrid", "naca4_polygon", "make_blade_grid", "blade_box_extent",
    "fourier_modes", "random_populations", "Workload", "RotorSpec",
    "workload", "WORKLOADS",
]
