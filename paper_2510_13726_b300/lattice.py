"""Python face of the C ABI: a lattice whose device memory comes from PyTorch.

Every step of the time loop runs in the library's CUDA kernels; this module
only allocates buffers with torch, passes pointers and sizes, and reshapes
results.  Arrays follow the lattice order (x fastest): fields have shape
(nz, ny, nx), vectors (3, nz, ny, nx).
"""

from __future__ import annotations

import ctypes as C

import numpy as np

from ._lib import LAYOUTS, STORAGE, HlConfig, HlRotorGeometry, check, lib

_ALIGN = 256


def _aligned_bytes(nbytes: int, device):
    import torch
    buf = torch.empty(int(nbytes) + _ALIGN, dtype=torch.uint8, device=device)
    off = (-buf.data_ptr()) % _ALIGN
    return buf, buf.data_ptr() + off


class Lattice:
    """A lattice with rotors, advanced on one CUDA stream of one device."""

    def __init__(self, nx, ny, nz, q=19, storage="f32", flow_axis=2, open_boundaries=True,
                 tau_mo=0.5005, c_smag=0.1, u_in=0.05, eps_h=2.0, transition="smoothstep",
                 sigma_band=1.0, wall_model=True, wm_E=9.8, wm_kappa=0.41, wm_ysample=2.0, wm_tol=1e-4,
                 wm_maxit=10, modes=None, mass_check_every=100, mass_tol=0.05, overlap=True,
                 layout="aa", halo_lo=False, halo_hi=False, z_offset=0, device=None, stream=None):
        import torch
        self.device = torch.device(device if device is not None else "cuda")
        if self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        L = lib()
        cfg = HlConfig()
        L.hl_config_defaults(C.byref(cfg))
        cfg.nx, cfg.ny, cfg.nz, cfg.q = int(nx), int(ny), int(nz), int(q)
        cfg.storage = STORAGE[storage] if isinstance(storage, str) else int(storage)
        cfg.flow_axis = int(flow_axis)
        cfg.open_boundaries = int(bool(open_boundaries))
        cfg.tau_mo, cfg.c_smag, cfg.u_in, cfg.eps_h = float(tau_mo), float(c_smag), float(u_in), float(eps_h)
        cfg.transition = 1 if transition == "linear" else 0
        cfg.sigma_band = float(sigma_band)
        cfg.wall_model = int(bool(wall_model))
        cfg.wm_E, cfg.wm_kappa, cfg.wm_ysample = float(wm_E), float(wm_kappa), float(wm_ysample)
        cfg.wm_tol, cfg.wm_maxit = float(wm_tol), int(wm_maxit)
        cfg.mass_check_every, cfg.mass_tol = int(mass_check_every), float(mass_tol)
        cfg.overlap = int(bool(overlap))
        cfg.layout = LAYOUTS[layout] if isinstance(layout, str) else int(layout)
        cfg.halo_lo, cfg.halo_hi, cfg.z_offset = int(halo_lo), int(halo_hi), int(z_offset)
        self._modes = None
        if modes is not None and len(modes):
            self._modes = np.ascontiguousarray(modes, dtype=np.float64).reshape(-1, 9)
            cfg.n_modes = self._modes.shape[0]
            cfg.modes = self._modes.ctypes.data_as(C.POINTER(C.c_double))
        self.cfg = cfg
        self.shape = (int(nz), int(ny), int(nx))
        self.N = int(nx) * int(ny) * int(nz)
        self.q = int(q)
        size = C.c_size_t()
        check(L.hl_workspace_size(C.byref(cfg), C.byref(size)))
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            self._ws, ptr = _aligned_bytes(size.value, self.device)
            h = C.c_void_p()
            check(L.hl_lattice_init(C.byref(h), C.byref(cfg), C.c_void_p(ptr), size.value,
                                    C.c_void_p(self.stream.cuda_stream)))
        self._h = h
        self._rotor_ws = []
        self.nrot = 0

    # -- lifetime -----------------------------------------------------------
    def close(self):
        """Release the handle and drop the device buffers it used."""
        if getattr(self, "_h", None):
            lib().hl_destroy(self._h)
            self._h = None
            self._ws = None
            self._rotor_ws = []

    def __del__(self):
        self.close()

    def _check(self, code):
        check(code, self._h)

    # -- rotors -------------------------------------------------------------
    def add_rotor(self, grid, center, omega, pitch=0.0, phase0=0.0, axis=None, n_blades=3,
                  hub_radius=None) -> int:
        """Add a rotor built from a ``workloads.BladeGrid`` (one blade, Sec. 3.1)."""
        import torch
        sdf = np.ascontiguousarray(grid.sdf, dtype=np.float32)
        g = HlRotorGeometry()
        g.center = (C.c_double * 3)(*[float(v) for v in center])
        g.axis = int(self.cfg.flow_axis if axis is None else axis)
        g.n_blades = int(n_blades)
        g.hub_radius = float(grid.hub_radius if hub_radius is None else hub_radius)
        g.phase0 = float(phase0)
        g.sdf = sdf.ctypes.data_as(C.POINTER(C.c_float))
        g.gz, g.gy, g.gx = sdf.shape
        g.origin = (C.c_double * 3)(*[float(v) for v in grid.origin])
        g.spacing = float(grid.spacing)
        size = C.c_size_t()
        self._check(lib().hl_rotor_workspace_size(self._h, C.byref(g), C.byref(size)))
        with torch.cuda.device(self.device):
            buf, ptr = _aligned_bytes(size.value, self.device)
            rid = C.c_int()
            self._check(lib().hl_set_rotor(self._h, C.byref(rid), C.byref(g), float(omega), float(pitch),
                                           C.c_void_p(ptr), size.value))
        self._rotor_ws.append(buf)
        self.nrot += 1
        return rid.value

    def rotor_box(self, k: int):
        lo = (C.c_int * 3)()
        n = (C.c_int * 3)()
        self._check(lib().hl_rotor_box(self._h, int(k), lo, n))
        return tuple(lo), tuple(n)

    def rotor_band(self, k: int):
        """Band arrays of the last porosity update, shaped (nbz, nby, nbx)."""
        import torch
        lo, n = self.rotor_box(k)
        box = n[0] * n[1] * n[2]
        dev = self.device
        d = torch.empty(box, dtype=torch.float32, device=dev)
        fl = torch.empty(box, dtype=torch.uint8, device=dev)
        wm = torch.empty(9 * box, dtype=torch.float32, device=dev)
        ut = torch.empty(box, dtype=torch.float64, device=dev)
        with torch.cuda.device(dev):
            self._check(lib().hl_rotor_band(self._h, int(k), d.data_ptr(), fl.data_ptr(), wm.data_ptr(),
                                            ut.data_ptr()))
        self.stream.synchronize()
        shp = (n[2], n[1], n[0])
        return dict(lo=lo, n=n, d=d.view(shp), flags=fl.view(shp), wm=wm.view((9,) + shp), utau=ut.view(shp))

    # -- time loop ----------------------------------------------------------
    def step(self, n: int = 1):
        import torch
        with torch.cuda.device(self.device):
            self._check(lib().hl_step(self._h, int(n)))

    # -- slabs (halo planes along z) -------------------------------------------
    def halo_size(self) -> int:
        """Bytes of one halo message (hl_halo_size)."""
        size = C.c_size_t()
        self._check(lib().hl_halo_size(self._h, C.byref(size)))
        return size.value

    def halo_export(self, face: int, buf):
        """Outgoing message of face 0 (lower) / 1 (upper) into the device tensor buf."""
        import torch
        with torch.cuda.device(self.device):
            self._check(lib().hl_halo_export(self._h, int(face), C.c_void_p(buf.data_ptr())))

    def halo_import(self, face: int, buf):
        """The neighbour's message for face 0 / 1 from the device tensor buf."""
        import torch
        with torch.cuda.device(self.device):
            self._check(lib().hl_halo_import(self._h, int(face), C.c_void_p(buf.data_ptr())))

    def halo_deep_size(self, face: int) -> int:
        """Bytes of the deep message of face 0 / 1 (hl_halo_deep_size)."""
        size = C.c_size_t()
        self._check(lib().hl_halo_deep_size(self._h, int(face), C.byref(size)))
        return size.value

    def halo_deep_export(self, face: int, buf):
        """Every slot of the slab's planes next to face 0 / 1 into the device tensor buf."""
        import torch
        with torch.cuda.device(self.device):
            self._check(lib().hl_halo_deep_export(self._h, int(face), C.c_void_p(buf.data_ptr())))

    def halo_deep_import(self, face: int, buf):
        """The neighbour's deep message for face 0 / 1 from the device tensor buf."""
        import torch
        with torch.cuda.device(self.device):
            self._check(lib().hl_halo_deep_import(self._h, int(face), C.c_void_p(buf.data_ptr())))

    def step_async(self, n: int = 1):
        import torch
        with torch.cuda.device(self.device):
            self._check(lib().hl_step_async(self._h, int(n)))

    def check(self):
        self._check(lib().hl_check(self._h))

    @property
    def t(self) -> int:
        v = C.c_longlong()
        self._check(lib().hl_get_time(self._h, C.byref(v)))
        return v.value

    # -- results ------------------------------------------------------------
    def forces(self, reset_avg: bool = False):
        """(F, F_avg): force on each rotor in the last step and its running mean, (nrot, 3)."""
        F = np.zeros((max(1, self.nrot), 3))
        Fa = np.zeros_like(F)
        self._check(lib().hl_forces(self._h, F.ctypes.data_as(C.POINTER(C.c_double)),
                                    Fa.ctypes.data_as(C.POINTER(C.c_double)), int(reset_avg)))
        return F[:self.nrot], Fa[:self.nrot]

    def loads_async(self, out):
        """Enqueue a copy of the last enqueued step's (F, M) per rotor into `out`, a pinned host
        float64 tensor of (nrot, 6) values, on the lattice stream; no synchronisation (record an
        event on self.stream after this call and wait for it before reading `out`)."""
        import torch
        if not (isinstance(out, torch.Tensor) and out.dtype == torch.float64 and not out.is_cuda
                and out.is_contiguous() and out.numel() >= 6 * self.nrot):
            raise ValueError("out must be a contiguous float64 host tensor of (nrot, 6) values")
        with torch.cuda.device(self.device):
            self._check(lib().hl_loads_async(self._h, out.data_ptr()))

    def moments(self):
        """(M, M_avg): torque about each rotor centre, (nrot, 3)."""
        M = np.zeros((max(1, self.nrot), 3))
        Ma = np.zeros_like(M)
        self._check(lib().hl_moments(self._h, M.ctypes.data_as(C.POINTER(C.c_double)),
                                     Ma.ctypes.data_as(C.POINTER(C.c_double))))
        return M[:self.nrot], Ma[:self.nrot]

    def fields(self):
        """Density (nz, ny, nx) and velocity (3, nz, ny, nx) as FP32 device tensors."""
        import torch
        rho = torch.empty(self.N, dtype=torch.float32, device=self.device)
        u = torch.empty(3 * self.N, dtype=torch.float32, device=self.device)
        with torch.cuda.device(self.device):
            self._check(lib().hl_fields(self._h, rho.data_ptr(), u.data_ptr()))
        self.stream.synchronize()
        return rho.view(self.shape), u.view((3,) + self.shape)

    def init_fields(self, rho=None, u=None):
        """Set f = f^eq(rho, u) from device tensors and reset t to 0."""
        import torch
        r = None if rho is None else torch.as_tensor(rho, dtype=torch.float32, device=self.device).contiguous()
        v = None if u is None else torch.as_tensor(u, dtype=torch.float32, device=self.device).contiguous()
        with torch.cuda.device(self.device):
            self._check(lib().hl_init_fields(self._h, 0 if r is None else r.data_ptr(),
                                             0 if v is None else v.data_ptr()))
        self.stream.synchronize()

    def mass(self) -> float:
        m = C.c_double()
        self._check(lib().hl_mass(self._h, C.byref(m)))
        return m.value

    # -- per-kernel timing ----------------------------------------------------
    KERNELS = ("band", "collide", "force", "mass", "wall", "collide_box")

    def profile_begin(self, capacity: int = 100000):
        self._check(lib().hl_profile_begin(self._h, int(capacity)))

    def profile_end(self):
        """{kernel: (total ms, launches)} of the launches since profile_begin."""
        ms = np.zeros(6)
        n = (C.c_longlong * 6)()
        self._check(lib().hl_profile_end(self._h, ms.ctypes.data_as(C.POINTER(C.c_double)), n))
        return {k: (float(ms[i]), int(n[i])) for i, k in enumerate(self.KERNELS)}

    # -- checkpoints --------------------------------------------------------
    def state_size(self) -> int:
        s = C.c_size_t()
        self._check(lib().hl_state_size(self._h, C.byref(s)))
        return s.value

    def save_state(self, buf=None):
        import torch
        n = self.state_size()
        if buf is None:
            buf = torch.empty(n, dtype=torch.uint8, device=self.device)
        with torch.cuda.device(self.device):
            self._check(lib().hl_save_state(self._h, buf.data_ptr(), buf.numel()))
        return buf

    def load_state(self, buf):
        import torch
        with torch.cuda.device(self.device):
            self._check(lib().hl_load_state(self._h, buf.data_ptr(), buf.numel()))

    # -- torque-driven rotors ---------------------------------------------------
    def set_drive(self, k: int, inertia: float, k_gen: float = 0.0, q_gen0: float = 0.0):
        """Rotor k turns under its aerodynamic torque from now on:
        I dOmega/dt = M.a - (q_gen0 + k_gen Omega |Omega|)."""
        self._check(lib().hl_set_drive(self._h, int(k), float(inertia), float(k_gen), float(q_gen0)))

    def drive_state(self, k: int):
        """(theta, Omega) of rotor k at the current step."""
        th, om = C.c_double(), C.c_double()
        self._check(lib().hl_drive_state(self._h, int(k), C.byref(th), C.byref(om)))
        return th.value, om.value

    def inflow_plane_shape(self):
        """(3, n_c, n_b) of the inlet plane: (b, c) = the axes after flow_axis, b fastest."""
        dims = (self.shape[2], self.shape[1], self.shape[0])
        a = self.cfg.flow_axis
        return (3, dims[(a + 2) % 3], dims[(a + 1) % 3])

    def set_inflow_plane(self, plane):
        """Inlet velocities from the caller: a device FP32 tensor of inflow_plane_shape(), read by
        every later step while set (overwrite it in place between steps on the lattice stream);
        None restores the synthetic inflow.  The tensor is kept alive by the lattice while set."""
        import torch
        if plane is None:
            self._inflow = None
            self._check(lib().hl_set_inflow_plane(self._h, None))
            return
        if not (isinstance(plane, torch.Tensor) and plane.is_cuda and plane.dtype == torch.float32
                and plane.is_contiguous() and tuple(plane.shape) == self.inflow_plane_shape()):
            raise ValueError(f"inflow plane must be a contiguous float32 device tensor of shape "
                             f"{self.inflow_plane_shape()}")
        self._inflow = plane
        self._check(lib().hl_set_inflow_plane(self._h, plane.data_ptr()))

    # -- gradients ------------------------------------------------------------
    def set_d0(self, d0):
        """Static porosity multiplier d0 (device tensor of N or (nz, ny, nx) floats; None = 1).
        The tensor is kept alive by the lattice while set."""
        import torch
        if d0 is None:
            self._d0 = None
            self._check(lib().hl_set_d0(self._h, None))
            return
        t = torch.as_tensor(d0, dtype=torch.float32, device=self.device).contiguous().view(-1)
        if t.numel() != self.N:
            raise ValueError("d0 must have one value per cell")
        self._d0 = t
        self._check(lib().hl_set_d0(self._h, t.data_ptr()))

    def set_pitch(self, k: int, pitch: float):
        self._check(lib().hl_set_pitch(self._h, int(k), float(pitch)))

    def freeze_sets(self, on: bool = True):
        """Hold the cell sets at the current pitches (finite-difference checks)."""
        self._check(lib().hl_freeze_sets(self._h, int(bool(on))))

    def grad_workspace_size(self, steps: int, ckpt_every: int) -> int:
        s = C.c_size_t()
        self._check(lib().hl_grad_workspace_size(self._h, int(steps), int(ckpt_every), C.byref(s)))
        return s.value

    def grad(self, steps: int, avg_last: int, w_thrust, w_torque, ckpt_every: int = 100, want_d0: bool = True,
             work=None):
        """Run `steps` steps and return (J, dJ/dpitch (nrot,), dJ/dd0 (nz, ny, nx) device tensor or None)
        for J = mean over the last avg_last steps of sum_k wT_k F_k.a_k + wQ_k M_k.a_k."""
        import torch
        wT = np.zeros(max(1, self.nrot))
        wQ = np.zeros(max(1, self.nrot))
        wT[:self.nrot] = w_thrust
        wQ[:self.nrot] = w_torque
        nbytes = self.grad_workspace_size(steps, ckpt_every)
        with torch.cuda.device(self.device):
            if work is None:
                buf, ptr = _aligned_bytes(nbytes, self.device)
            else:
                buf, ptr = work, work.data_ptr()
                if ptr % _ALIGN or work.numel() * work.element_size() < nbytes:
                    raise ValueError("gradient workspace too small or not 256-byte aligned")
            gd0 = torch.empty(self.N, dtype=torch.float32, device=self.device) if want_d0 else None
            J = C.c_double()
            gp = np.zeros(max(1, self.nrot))
            self._check(lib().hl_grad(self._h, int(steps), int(avg_last), int(ckpt_every),
                                      wT.ctypes.data_as(C.POINTER(C.c_double)),
                                      wQ.ctypes.data_as(C.POINTER(C.c_double)), C.byref(J),
                                      gp.ctypes.data_as(C.POINTER(C.c_double)),
                                      None if gd0 is None else gd0.data_ptr(), C.c_void_p(ptr), nbytes))
        del buf
        return J.value, gp[:self.nrot], (None if gd0 is None else gd0.view(self.shape))

    @classmethod
    def from_workload(cls, wl, storage="f32", q=None, rotor_kw=None, **overrides):
        """Lattice and rotors of a ``workloads.Workload``."""
        kw = dict(q=wl.q if q is None else q, storage=storage, flow_axis=wl.flow_axis,
                  tau_mo=wl.tau_mo, c_smag=wl.c_smag, u_in=wl.u_in, eps_h=wl.eps_h, modes=wl.modes())
        kw.update(overrides)
        lat = cls(wl.nx, wl.ny, wl.nz, **kw)
        for spec, g in zip(wl.rotors, wl.blade_grids()):
            rk = dict(center=spec.center, omega=spec.omega(wl.u_in), pitch=spec.pitch,
                      phase0=spec.phase0, n_blades=spec.n_blades)
            if rotor_kw:
                rk.update(rotor_kw)
            lat.add_rotor(g, **rk)
        return lat
