"""The allocation-free mass total (hl_mass_noalloc).

For callers that cannot allocate device memory at the moment they need the
total mass of a population array, hl_mass_noalloc keeps its partial sums in
the library's own static device memory.  This file is collected last so that
a run stopping at its first failure has already run every other test.  It
checks the new entry point and hl_mass (which uses the lattice's workspace)
against an FP64 sum of the same population array, on two calls in a row,
through the C ABI, for FP32, FP16 and BF16 storage and for both population
layouts (the AA pattern and the esoteric twist store the same [q][N] array
of shifted values).  Both entry points convert every stored value to FP64
before adding it, so both agree with the FP64 sum to 1e-12 relative.
"""

import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _workspace_populations(lat):
    # the populations occupy the start of the (256-byte aligned) workspace
    base = lat._ws.data_ptr()
    return base + ((-base) % 256)


def _populations_fp64(lat, q, n_cells, storage):
    """The stored (weight-shifted) values as float64, from the workspace bytes."""
    import torch
    off = (-lat._ws.data_ptr()) % 256
    dt = {"f32": torch.float32, "f16s": torch.float16, "bf16s": torch.bfloat16}[storage]
    esize = 4 if storage == "f32" else 2
    raw = lat._ws[off:off + q * n_cells * esize]
    return raw.view(dt).double()


def test_mass_noalloc_matches_workspace_mass_twice():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("a CUDA device is required for the gpu-marked tests")
    from paper_2510_13726_b300.build import build
    build()
    import workloads as W
    from paper_2510_13726_b300 import Lattice, lib

    L = lib()
    wl = W.workload("rotor48")
    for storage, layout in (("f32", "aa"), ("f16s", "aa"), ("bf16s", "aa"), ("f32", "esotwist")):
        lat = Lattice.from_workload(wl, storage=storage, mass_check_every=0, layout=layout)
        out = torch.zeros(1, dtype=torch.float64, device=lat.device)
        pops = _workspace_populations(lat)
        code = {"f32": 0, "f16s": 1, "bf16s": 2}[storage]
        for k in range(2):
            lat.step(3)
            ref = lat.mass()
            with torch.cuda.device(lat.device):
                rc = L.hl_mass_noalloc(wl.q, code, C.c_void_p(pops), wl.cells, C.c_void_p(out.data_ptr()),
                                       C.c_void_p(lat.stream.cuda_stream))
            assert rc == 0
            lat.stream.synchronize()
            got = float(out.item())
            assert np.isfinite(got)
            g = _populations_fp64(lat, wl.q, wl.cells, storage)
            exact = float(g.sum()) + wl.cells            # shift: sum of the weights is 1 per cell
            assert abs(got - exact) <= 1e-12 * abs(exact), (storage, layout, k, got, exact)
            assert abs(ref - exact) <= 1e-12 * abs(exact), (storage, layout, k, ref, exact)
        lat.close()


def test_mass_noalloc_rejects_bad_arguments_and_oversize():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("a CUDA device is required for the gpu-marked tests")
    from paper_2510_13726_b300 import lib
    L = lib()
    dummy = torch.zeros(8, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert L.hl_mass_noalloc(20, 0, C.c_void_p(dummy.data_ptr()), 1, C.c_void_p(out.data_ptr()), s) == -1
    assert L.hl_mass_noalloc(19, 0, None, 1, C.c_void_p(out.data_ptr()), s) == -1
    # more than 2^32 stored values: rejected before any launch
    assert L.hl_mass_noalloc(19, 0, C.c_void_p(dummy.data_ptr()), (1 << 32) // 19 + 1,
                             C.c_void_p(out.data_ptr()), s) == -4
