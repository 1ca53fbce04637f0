"""B300 (sm_103a) homogenized lattice Boltzmann rotor library.

Hot path: hand-written CUDA kernels behind the C ABI ``include/hlbm.h``
(``libhlbm.so``).  This package is the thin binding: argument marshalling
through ctypes, with PyTorch supplying device memory and streams.  There is
no CPU fallback: loading fails loudly when the CUDA library is missing.
"""

from ._lib import HlConfig, HlRotorGeometry, HlError, lib, velocity_set
from .lattice import Lattice
from .objective import rotor_objective

__all__ = ["HlConfig", "HlRotorGeometry", "HlError", "lib", "velocity_set", "Lattice", "rotor_objective"]
