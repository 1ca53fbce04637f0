"""ctypes binding of the C ABI in include/hlbm.h (argument marshalling only)."""

from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIBPATH = os.path.join(HERE, "libhlbm.so")

HL_OK = 0
STATUS = {0: "HL_OK", -1: "HL_ERR_ARG", -2: "HL_ERR_CUDA", -3: "HL_ERR_NONFINITE",
          -4: "HL_ERR_WORKSPACE", -5: "HL_ERR_STATE", -8: "HL_ERR_MASS", -9: "HL_ERR_GEOMETRY"}
STORAGE = {"f32": 0, "f16s": 1, "bf16s": 2}
# population layouts: AA pattern, esoteric twist, AA pattern with each x row stored as interleaved halves
LAYOUTS = {"aa": 0, "esotwist": 1, "aa_halves": 2}

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)
_vp = C.c_void_p


class HlConfig(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("q", C.c_int), ("storage", C.c_int),
        ("flow_axis", C.c_int), ("open_boundaries", C.c_int),
        ("tau_mo", C.c_double), ("c_smag", C.c_double), ("u_in", C.c_double),
        ("sigma_band", C.c_double), ("eps_h", C.c_double),
        ("transition", C.c_int), ("wall_model", C.c_int),
        ("wm_E", C.c_double), ("wm_kappa", C.c_double), ("wm_ysample", C.c_double),
        ("wm_tol", C.c_double), ("wm_maxit", C.c_int),
        ("n_modes", C.c_int), ("modes", _dp),
        ("mass_check_every", C.c_int), ("mass_tol", C.c_double), ("overlap", C.c_int),
        ("layout", C.c_int), ("halo_lo", C.c_int), ("halo_hi", C.c_int), ("z_offset", C.c_int),
    ]


class HlRotorGeometry(C.Structure):
    _fields_ = [
        ("center", C.c_double * 3), ("axis", C.c_int), ("n_blades", C.c_int),
        ("hub_radius", C.c_double), ("phase0", C.c_double), ("sdf", C.POINTER(C.c_float)),
        ("gx", C.c_int), ("gy", C.c_int), ("gz", C.c_int), ("origin", C.c_double * 3),
        ("spacing", C.c_double),
    ]


class HlError(RuntimeError):
    def __init__(self, code, msg=""):
        self.code = code
        super().__init__(f"{STATUS.get(code, code)}: {msg}")


# name -> (restype, argtypes); every symbol declared in include/hlbm.h
SIGNATURES = {
    "hl_config_defaults": (None, [C.POINTER(HlConfig)]),
    "hl_workspace_size": (C.c_int, [C.POINTER(HlConfig), C.POINTER(C.c_size_t)]),
    "hl_lattice_init": (C.c_int, [C.POINTER(_vp), C.POINTER(HlConfig), _vp, C.c_size_t, _vp]),
    "hl_rotor_workspace_size": (C.c_int, [_vp, C.POINTER(HlRotorGeometry), C.POINTER(C.c_size_t)]),
    "hl_set_rotor": (C.c_int, [_vp, _ip, C.POINTER(HlRotorGeometry), C.c_double, C.c_double, _vp,
                               C.c_size_t]),
    "hl_step": (C.c_int, [_vp, C.c_int]),
    "hl_step_async": (C.c_int, [_vp, C.c_int]),
    "hl_check": (C.c_int, [_vp]),
    "hl_forces": (C.c_int, [_vp, _dp, _dp, C.c_int]),
    "hl_moments": (C.c_int, [_vp, _dp, _dp]),
    "hl_fields": (C.c_int, [_vp, _vp, _vp]),
    "hl_init_fields": (C.c_int, [_vp, _vp, _vp]),
    "hl_mass": (C.c_int, [_vp, _dp]),
    "hl_get_time": (C.c_int, [_vp, C.POINTER(C.c_longlong)]),
    "hl_state_size": (C.c_int, [_vp, C.POINTER(C.c_size_t)]),
    "hl_save_state": (C.c_int, [_vp, _vp, C.c_size_t]),
    "hl_load_state": (C.c_int, [_vp, _vp, C.c_size_t]),
    "hl_rotor_box": (C.c_int, [_vp, C.c_int, _ip, _ip]),
    "hl_rotor_band": (C.c_int, [_vp, C.c_int, _vp, _vp, _vp, _vp]),
    "hl_velocity_set": (C.c_int, [C.c_int, _ip, _dp]),
    "hl_debug_collide": (C.c_int, [C.c_int, C.c_int, _vp, _vp, _vp, _vp, _vp, C.c_double, C.c_double,
                                   _vp, _vp]),
    "hl_set_drive": (C.c_int, [_vp, C.c_int, C.c_double, C.c_double, C.c_double]),
    "hl_drive_state": (C.c_int, [_vp, C.c_int, _dp, _dp]),
    "hl_set_d0": (C.c_int, [_vp, _vp]),
    "hl_set_inflow_plane": (C.c_int, [_vp, _vp]),
    "hl_loads_async": (C.c_int, [_vp, _vp]),
    "hl_debug_collide_pair": (C.c_int, [C.c_int, C.c_int, _vp, C.c_double, C.c_double, _vp, _vp]),
    "hl_set_pitch": (C.c_int, [_vp, C.c_int, C.c_double]),
    "hl_freeze_sets": (C.c_int, [_vp, C.c_int]),
    "hl_grad_workspace_size": (C.c_int, [_vp, C.c_int, C.c_int, C.POINTER(C.c_size_t)]),
    "hl_grad": (C.c_int, [_vp, C.c_int, C.c_int, C.c_int, _dp, _dp, _dp, _dp, _vp, _vp, C.c_size_t]),
    "hl_debug_collide_vjp": (C.c_int, [C.c_int, C.c_int, _vp, _vp, _vp, _vp, _vp, C.c_double, C.c_double,
                                       _vp, _vp, _vp, _vp, _vp, _vp]),
    "hl_profile_begin": (C.c_int, [_vp, C.c_int]),
    "hl_profile_end": (C.c_int, [_vp, _dp, C.POINTER(C.c_longlong)]),
    "hl_mass_noalloc": (C.c_int, [C.c_int, C.c_int, _vp, C.c_longlong, _vp, _vp]),
    "hl_halo_size": (C.c_int, [_vp, C.POINTER(C.c_size_t)]),
    "hl_halo_export": (C.c_int, [_vp, C.c_int, _vp]),
    "hl_halo_import": (C.c_int, [_vp, C.c_int, _vp]),
    "hl_halo_deep_size": (C.c_int, [_vp, C.c_int, C.POINTER(C.c_size_t)]),
    "hl_halo_deep_export": (C.c_int, [_vp, C.c_int, _vp]),
    "hl_halo_deep_import": (C.c_int, [_vp, C.c_int, _vp]),
    "hl_last_error": (C.c_char_p, [_vp]),
    "hl_destroy": (None, [_vp]),
}

_LIB = None


def lib():
    """Load libhlbm.so (raises if it has not been built: there is no fallback)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIBPATH):
            raise RuntimeError(f"CUDA library not built: {LIBPATH} (run python -m paper_2510_13726_b300.build)")
        L = C.CDLL(LIBPATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = L
    return _LIB


def check(code, handle=None):
    if code != HL_OK:
        msg = ""
        if handle:
            m = lib().hl_last_error(handle)
            msg = m.decode() if m else ""
        raise HlError(code, msg)


def velocity_set(q: int):
    """(c[q][3], w[q]) in the library's slot order."""
    c = np.zeros((q, 3), dtype=np.int32)
    w = np.zeros(q)
    check(lib().hl_velocity_set(q, c.ctypes.data_as(_ip), w.ctypes.data_as(_dp)))
    return c.astype(np.int64), w
