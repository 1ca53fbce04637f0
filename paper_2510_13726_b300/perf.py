"""Algorithmic traffic model of the time step (used for the roofline).

The fused collide-and-stream kernel reads and writes every population once
per cell update (AA pattern, single buffer): 2 q s bytes per cell, s the
storage size (4 for FP32, 2 for FP16/BF16 shifted storage).  This is the
paper's count of 152 bytes per RRLBM D3Q19 cell update (Sec. 5, Table).
Cells in a rotor box additionally read the porosity (4 B) and flags (1 B);
wall cells read the modelled velocity and strain (9 x 4 B).
"""

STORE_BYTES = {"f32": 4, "f16s": 2, "bf16s": 2}


def bytes_per_cell(q: int, storage: str = "f32") -> int:
    return 2 * q * STORE_BYTES[storage]


def collide_bytes(q: int, storage: str, cells: int, box_cells: int = 0, wall_cells: int = 0) -> int:
    """Algorithmic bytes of one collide-and-stream launch."""
    return bytes_per_cell(q, storage) * cells + 5 * box_cells + 36 * wall_cells
