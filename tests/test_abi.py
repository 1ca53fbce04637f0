"""Host-side checks of the C ABI (no GPU): the library builds and loads,
exports every symbol include/hlbm.h declares, and validates arguments."""

import ctypes as C
import os
import re

import numpy as np
import pytest

import oracle as O
from paper_2510_13726_b300 import _lib
from paper_2510_13726_b300.build import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    build()
    return _lib.lib()


def _declared():
    txt = open(os.path.join(ROOT, "include", "hlbm.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(hl_[a-z0-9_]+)\s*\(", txt)))


def test_every_declared_symbol_is_exported_and_bound(L):
    names = _declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(_lib.SIGNATURES)


def test_struct_layouts_match_header():
    # field order and count mirror include/hlbm.h
    txt = open(os.path.join(ROOT, "include", "hlbm.h")).read()
    body = txt[txt.index("typedef struct hl_config {"):txt.index("} hl_config;")]
    fields = re.findall(r"\b(\w+)\s*[,;]", re.sub(r"/\*.*?\*/", "", body, flags=re.S))
    names = [f[0] for f in _lib.HlConfig._fields_]
    assert [f for f in fields if f in names] == names


def test_defaults_and_workspace_size(L):
    cfg = _lib.HlConfig()
    L.hl_config_defaults(C.byref(cfg))
    assert cfg.q == 19 and cfg.wm_E == 9.8 and cfg.wm_kappa == 0.41 and cfg.wm_maxit == 10
    size = C.c_size_t()
    assert L.hl_workspace_size(C.byref(cfg), C.byref(size)) == -1      # grid size not set
    cfg.nx, cfg.ny, cfg.nz = 48, 48, 96
    assert L.hl_workspace_size(C.byref(cfg), C.byref(size)) == 0
    N = 48 * 48 * 96
    assert size.value >= 19 * N * 4
    assert size.value < 19 * N * 4 + 4 * 1024 * 1024
    cfg.storage = 2
    s16 = C.c_size_t()
    assert L.hl_workspace_size(C.byref(cfg), C.byref(s16)) == 0
    assert s16.value < size.value
    for bad in (dict(q=20), dict(storage=5), dict(flow_axis=3), dict(tau_mo=0.5), dict(nx=1),
                dict(sigma_band=1.5), dict(sigma_band=-0.25), dict(mass_check_every=-1), dict(layout=3),
                dict(layout=2, nx=47), dict(layout=1, halo_hi=1)):
        c2 = _lib.HlConfig()
        L.hl_config_defaults(C.byref(c2))
        c2.nx, c2.ny, c2.nz = 48, 48, 96
        for k, v in bad.items():
            setattr(c2, k, v)
        assert L.hl_workspace_size(C.byref(c2), C.byref(size)) == -1, bad
    # the AA layout with x halves: nx even, slabs allowed
    for good in (dict(layout=2), dict(layout=2, halo_lo=1, halo_hi=1)):
        c2 = _lib.HlConfig()
        L.hl_config_defaults(C.byref(c2))
        c2.nx, c2.ny, c2.nz = 48, 48, 96
        for k, v in good.items():
            setattr(c2, k, v)
        assert L.hl_workspace_size(C.byref(c2), C.byref(size)) == 0, good


def test_bytes_per_cell_match_paper_table(golden):
    """Sec. 5, Table: RRLBM D3Q19 moves 152 bytes per cell update, i.e. one
    read and one write of 19 FP32 populations: the library's byte model."""
    from paper_2510_13726_b300.perf import bytes_per_cell
    assert bytes_per_cell(19, "f32") == golden["bytes_per_cell_rrlbm_d3q19"]["value"]
    assert bytes_per_cell(27, "f32") == 216
    assert bytes_per_cell(27, "bf16s") == 108


@pytest.mark.parametrize("q", [19, 27])
def test_velocity_set_matches_oracle_as_a_set(q):
    c, w = _lib.velocity_set(q)
    co, wo, _ = O.lattice(q)
    a = {tuple(v): x for v, x in zip(c, w)}
    b = {tuple(v): x for v, x in zip(co, wo)}
    assert a == b
    # slot order: rest, P positives, then their opposites
    P = (q - 1) // 2
    assert np.all(c[0] == 0)
    assert np.all(c[1:1 + P] == -c[1 + P:])


def test_null_and_invalid_handles_are_rejected(L):
    assert L.hl_step(None, 1) == -1
    assert L.hl_check(None) == -1
    assert L.hl_forces(None, None, None, 0) == -1
    assert L.hl_last_error(None) == b"null handle"
    assert L.hl_debug_collide(20, 1, None, None, None, None, None, 0.6, 0.1, None, None) == -1


def test_slab_configuration_rules(L):
    """Halo planes (0 to 8 per face) need an AA layout and at least as many
    owned planes as either face has halo planes (the deep message of a face
    is the slab's own planes next to it); a periodic slab may start at
    z_offset -1 (host-side validation only)."""
    cfg = _lib.HlConfig()
    L.hl_config_defaults(C.byref(cfg))
    cfg.nx, cfg.ny, cfg.nz = 8, 8, 6
    size = C.c_size_t()
    assert L.hl_workspace_size(C.byref(cfg), C.byref(size)) == 0
    plain = size.value
    cfg.halo_lo, cfg.halo_hi, cfg.z_offset = 1, 1, -1
    assert L.hl_workspace_size(C.byref(cfg), C.byref(size)) == 0 and size.value == plain
    cfg.layout = 1
    assert L.hl_workspace_size(C.byref(cfg), C.byref(size)) == -1      # slabs use the AA pattern
    cfg.layout = 2
    assert L.hl_workspace_size(C.byref(cfg), C.byref(size)) == 0       # the AA layout with x halves
    cfg.layout = 0
    cfg.halo_lo = 2                                                     # 2 + 1 halo planes, 3 owned
    assert L.hl_workspace_size(C.byref(cfg), C.byref(size)) == 0
    cfg.halo_lo = 4                                                     # 4 + 1 halo planes, 1 owned
    assert L.hl_workspace_size(C.byref(cfg), C.byref(size)) == -1
    cfg.nz, cfg.halo_lo, cfg.halo_hi = 20, 9, 1
    assert L.hl_workspace_size(C.byref(cfg), C.byref(size)) == -1      # at most 8
    cfg.halo_lo, cfg.halo_hi = -1, 1
    assert L.hl_workspace_size(C.byref(cfg), C.byref(size)) == -1
    cfg.halo_lo, cfg.halo_hi, cfg.nz = 1, 1, 2
    assert L.hl_workspace_size(C.byref(cfg), C.byref(size)) == -1      # nz < 3
