"""FP64 CPU oracle of the HHRRLBM-LES rotor scheme -- TEST INFRASTRUCTURE.

Plain, slow, obviously-correct statement of what the CUDA library computes
(arXiv 2510.13726, Sec. 2-3), written in C (``hlbm_oracle.c``) and loaded
through ctypes.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference leg of ``bench.py`` may import this package.
It shares no code with ``paper_2510_13726_b300``; both take their inputs from
``workloads`` (seeded data only).

Parity status of each part (the pins live in ``tests/test_oracle_*.py``):
  lattice, equilibrium, regularized non-equilibrium, Smagorinsky tau,
  collision, wall function, porosity definition, embedding, streaming,
  invariants: pinned; wall model of a wall cell (sample point, tangential
  relative velocity, friction velocity at the sample's wall distance,
  modelled velocity u_tau u+(y1+), strain, Newton start values): pinned in
  the log-law regime against closed forms on flat walls and by a log-law
  channel; open boundaries: pinned by a uniform stream (fixed point) and a
  parallel shear flow leaving through the outlet; boundary force (momentum
  exchange): pinned against the momentum deficit and symmetry; physical
  accuracy on the paper's rotor (C_T ~ 0.963): parity unpinned (geometry and
  data are not available).
"""

from __future__ import annotations

import ctypes as C

import numpy as np

from . import build as _build

_LIB = None

_dp = C.POINTER(C.c_double)
_fp = C.POINTER(C.c_float)
_ip = C.POINTER(C.c_int)
_u8p = C.POINTER(C.c_uint8)
_i8p = C.POINTER(C.c_int8)


class Params(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("q", C.c_int),
        ("flow_axis", C.c_int), ("open_boundaries", C.c_int),
        ("tau_mo", C.c_double), ("c_smag", C.c_double), ("u_in", C.c_double),
        ("sigma_band", C.c_double), ("eps_h", C.c_double),
        ("transition", C.c_int), ("wall_model", C.c_int),
        ("wm_E", C.c_double), ("wm_kappa", C.c_double), ("wm_ysample", C.c_double),
        ("wm_tol", C.c_double), ("wm_maxit", C.c_int), ("force_form", C.c_int),
        ("n_modes", C.c_int), ("modes", _dp),
    ]


class Rotor(C.Structure):
    _fields_ = [
        ("center", C.c_double * 3), ("axis", C.c_int), ("n_blades", C.c_int),
        ("hub_radius", C.c_double), ("phase0", C.c_double), ("omega", C.c_double),
        ("pitch", C.c_double), ("sdf", _fp), ("gx", C.c_int), ("gy", C.c_int),
        ("gz", C.c_int), ("origin", C.c_double * 3), ("spacing", C.c_double),
    ]


def lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        L = C.CDLL(path)
        L.or_create.restype = C.c_void_p
        L.or_create.argtypes = [C.POINTER(Params), C.POINTER(Rotor), C.c_int]
        L.or_destroy.argtypes = [C.c_void_p]
        L.or_step.argtypes = [C.c_void_p, C.c_int]
        L.or_time.restype = C.c_long
        L.or_time.argtypes = [C.c_void_p]
        L.or_get_populations.argtypes = [C.c_void_p, _dp]
        L.or_set_populations.argtypes = [C.c_void_p, _dp]
        L.or_init_equilibrium.argtypes = [C.c_void_p, _dp, _dp]
        L.or_fields.argtypes = [C.c_void_p, _dp, _dp]
        L.or_forces.argtypes = [C.c_void_p, _dp, _dp, _dp, _dp]
        L.or_reset_average.argtypes = [C.c_void_p]
        L.or_mass.restype = C.c_double
        L.or_mass.argtypes = [C.c_void_p]
        L.or_geometry.argtypes = [C.c_void_p, _fp, _dp, _u8p, _i8p]
        L.or_wall_state.argtypes = [C.c_void_p, _dp, _dp, _dp, _u8p, _dp]
        L.or_newton_stats.argtypes = [C.c_void_p, C.POINTER(C.c_long), C.POINTER(C.c_long)]
        L.or_inflow_plane.argtypes = [C.c_void_p, C.c_long, _dp]
        L.or_lattice_table.restype = C.c_int
        L.or_lattice_table.argtypes = [C.c_int, _ip, _dp, _ip]
        L.or_equilibrium.restype = C.c_int
        L.or_equilibrium.argtypes = [C.c_int, C.c_double, _dp, _dp]
        L.or_regularized_neq.restype = C.c_int
        L.or_regularized_neq.argtypes = [C.c_int, _dp, _dp, _dp]
        L.or_smagorinsky_tau.restype = C.c_double
        L.or_smagorinsky_tau.argtypes = [C.c_double, C.c_double, C.c_double, _dp]
        L.or_collide_cells.restype = C.c_int
        L.or_collide_cells.argtypes = [C.c_int, C.c_int, _dp, _dp, _dp, _dp, _dp,
                                       C.c_double, C.c_double, _dp, _dp]
        L.or_spalding_yplus.restype = C.c_double
        L.or_spalding_yplus.argtypes = [C.c_double, C.c_double, C.c_double]
        L.or_spalding_uplus.restype = C.c_double
        L.or_spalding_uplus.argtypes = [C.c_double, C.c_double, C.c_double, C.c_double, C.c_int]
        L.or_wall_newton.restype = C.c_double
        L.or_wall_newton.argtypes = [C.c_double, C.c_double, C.c_double, C.c_double,
                                     C.c_double, C.c_double, C.c_double, C.c_int, _ip]
        L.or_porosity.restype = C.c_double
        L.or_porosity.argtypes = [C.c_double, C.c_double, C.c_int]
        L.or_rotor_phi.argtypes = [C.POINTER(Rotor), C.c_long, C.c_int, _ip, _fp, _ip]
        L.or_rotor_normal.argtypes = [C.POINTER(Rotor), C.c_long, C.c_int, C.c_int, C.c_int,
                                      C.c_int, _dp]
        L.or_collide_vjp_cells.restype = C.c_int
        L.or_collide_vjp_cells.argtypes = [C.c_int, C.c_int, _dp, _dp, _dp, _dp, _dp, C.c_double,
                                           C.c_double, _dp, _dp, _dp, _dp, _dp]
        L.or_set_d0.restype = C.c_int
        L.or_set_d0.argtypes = [C.c_void_p, _dp]
        L.or_set_pitch.restype = C.c_int
        L.or_set_pitch.argtypes = [C.c_void_p, C.c_int, C.c_double]
        L.or_freeze_sets.argtypes = [C.c_void_p, C.c_int]
        L.or_adjoint.restype = C.c_int
        L.or_adjoint.argtypes = [C.c_void_p, C.c_int, C.c_int, _dp, _dp, _dp, _dp, _dp]
        L.or_set_drive.restype = C.c_int
        L.or_set_drive.argtypes = [C.c_void_p, C.c_int, C.c_double, C.c_double, C.c_double]
        L.or_drive_state.restype = C.c_int
        L.or_drive_state.argtypes = [C.c_void_p, C.c_int, _dp, _dp]
        L.or_porosity_tangent.argtypes = [C.c_void_p, _dp]
        L.or_fd_strain.argtypes = [C.c_void_p, _dp]
        L.or_wall_tangent.argtypes = [C.c_void_p, _dp, _dp]
        L.or_rotor_normal_tangent.argtypes = [C.POINTER(Rotor), C.c_long, C.c_int, C.c_int, C.c_int,
                                              C.c_int, _dp]
        L.or_sizeof_params.restype = C.c_size_t
        L.or_sizeof_rotor.restype = C.c_size_t
        assert L.or_sizeof_params() == C.sizeof(Params)
        assert L.or_sizeof_rotor() == C.sizeof(Rotor)
        _LIB = L
    return _LIB


def _ptr(a, t=_dp):
    return a.ctypes.data_as(t) if a is not None else None


def lattice(q: int):
    """Velocities c[q][3], weights w[q], opposite index opp[q] of the oracle's D3Q19/D3Q27."""
    c = np.zeros((q, 3), dtype=np.int32)
    w = np.zeros(q)
    opp = np.zeros(q, dtype=np.int32)
    if lib().or_lattice_table(q, _ptr(c, _ip), _ptr(w), _ptr(opp, _ip)):
        raise ValueError("q must be 19 or 27")
    return c.astype(np.int64), w, opp.astype(np.int64)


def equilibrium(q: int, rho: float, u) -> np.ndarray:
    u = np.ascontiguousarray(u, dtype=np.float64)
    out = np.zeros(q)
    lib().or_equilibrium(q, float(rho), _ptr(u), _ptr(out))
    return out


def regularized_neq(q: int, a2, u) -> np.ndarray:
    a2 = np.ascontiguousarray(a2, dtype=np.float64).reshape(9)
    u = np.ascontiguousarray(u, dtype=np.float64)
    out = np.zeros(q)
    lib().or_regularized_neq(q, _ptr(a2), _ptr(u), _ptr(out))
    return out


def smagorinsky_tau(tau_mo: float, c_smag: float, rho: float, pneq) -> float:
    p = np.ascontiguousarray(pneq, dtype=np.float64).reshape(9)
    return lib().or_smagorinsky_tau(tau_mo, c_smag, rho, _ptr(p))


def collide_cells(q, f, d=None, uB=None, sigma=None, Sfd=None, tau_mo=0.5005, c_smag=0.1):
    """Collide n independent cells: f[n][q] -> (f*[n][q], tau_eff[n])."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    n = f.shape[0]

    def conv(a, s):
        if a is None:
            return None
        return np.ascontiguousarray(np.broadcast_to(np.asarray(a, dtype=np.float64), s))

    d = conv(d, (n,))
    uB = conv(uB, (n, 3))
    sigma = conv(sigma, (n,))
    Sfd = conv(Sfd, (n, 3, 3))
    out = np.zeros_like(f)
    tau = np.zeros(n)
    lib().or_collide_cells(q, n, _ptr(f), _ptr(d), _ptr(uB), _ptr(sigma), _ptr(Sfd),
                           tau_mo, c_smag, _ptr(out), _ptr(tau))
    return out, tau


def spalding_yplus(up, E=9.8, kappa=0.41):
    return lib().or_spalding_yplus(float(up), E, kappa)


def spalding_uplus(yp, E=9.8, kappa=0.41, tol=1e-4, maxit=10):
    return lib().or_spalding_uplus(float(yp), E, kappa, tol, maxit)


def wall_newton(u, y, nu, guess, E=9.8, kappa=0.41, tol=1e-4, maxit=10):
    it = C.c_int(0)
    r = lib().or_wall_newton(float(u), float(y), float(nu), float(guess), E, kappa, tol, maxit,
                             C.byref(it))
    return r, it.value


def porosity(phi, eps=2.0, linear=False):
    return lib().or_porosity(float(phi), float(eps), int(linear))


def make_rotor(grid, center, axis=2, omega=0.0, phase0=0.0, pitch=0.0, n_blades=3,
               hub_radius=None):
    """ctypes rotor description; keeps a reference to the float32 grid."""
    sdf = np.ascontiguousarray(grid.sdf, dtype=np.float32)
    r = Rotor()
    r.center = (C.c_double * 3)(*[float(v) for v in center])
    r.axis = int(axis)
    r.n_blades = int(n_blades)
    r.hub_radius = float(grid.hub_radius if hub_radius is None else hub_radius)
    r.phase0 = float(phase0)
    r.omega = float(omega)
    r.pitch = float(pitch)
    r.sdf = _ptr(sdf, _fp)
    gz, gy, gx = sdf.shape
    r.gx, r.gy, r.gz = gx, gy, gz
    r.origin = (C.c_double * 3)(*[float(v) for v in grid.origin])
    r.spacing = float(grid.spacing)
    r._keep = sdf
    return r


def rotor_phi(rotor, t, xyz):
    xyz = np.ascontiguousarray(xyz, dtype=np.int32).reshape(-1, 3)
    n = xyz.shape[0]
    phi = np.zeros(n, dtype=np.float32)
    which = np.zeros(n, dtype=np.int32)
    lib().or_rotor_phi(C.byref(rotor), int(t), n, _ptr(xyz, _ip), _ptr(phi, _fp), _ptr(which, _ip))
    return phi, which


def rotor_normal_tangent(rotor, t, which, x, y, z):
    """d n / d pitch of component `which` at cell (x, y, z), time t (complex step)."""
    dn = np.zeros(3)
    lib().or_rotor_normal_tangent(C.byref(rotor), int(t), int(which), int(x), int(y), int(z), _ptr(dn))
    return dn


def rotor_normal(rotor, t, which, x, y, z):
    n = np.zeros(3)
    lib().or_rotor_normal(C.byref(rotor), int(t), int(which), int(x), int(y), int(z), _ptr(n))
    return n


def collide_vjp_cells(q, f, lam_star, d=None, uB=None, sigma=None, Sfd=None, tau_mo=0.5005, c_smag=0.1):
    """Vector-Jacobian product of the collision of n independent cells, by
    complex-step differentiation: lam_star[n][q] (adjoint of f*) ->
    (lam_f[n][q], g_d[n], g_uB[n][3], g_S[n][3][3])."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    lam_star = np.ascontiguousarray(lam_star, dtype=np.float64).reshape(f.shape)
    n = f.shape[0]

    def conv(a, s):
        if a is None:
            return None
        return np.ascontiguousarray(np.broadcast_to(np.asarray(a, dtype=np.float64), s))

    d = conv(d, (n,))
    uB = conv(uB, (n, 3))
    sigma = conv(sigma, (n,))
    Sfd = conv(Sfd, (n, 3, 3))
    lam_f = np.zeros_like(f)
    g_d = np.zeros(n)
    g_uB = np.zeros((n, 3))
    g_S = np.zeros((n, 3, 3))
    rc = lib().or_collide_vjp_cells(q, n, _ptr(f), _ptr(d), _ptr(uB), _ptr(sigma), _ptr(Sfd), tau_mo, c_smag,
                                    _ptr(lam_star), _ptr(lam_f), _ptr(g_d), _ptr(g_uB), _ptr(g_S))
    if rc:
        raise ValueError("oracle: bad lattice")
    return lam_f, g_d, g_uB, g_S


class Oracle:
    """Whole-lattice FP64 reference run.

    Arrays follow the lattice order (x fastest): fields are returned with
    shape (nz, ny, nx); populations with shape (q, nz, ny, nx).
    """

    def __init__(self, nx, ny, nz, q=19, flow_axis=2, open_boundaries=True, tau_mo=0.5005,
                 c_smag=0.1, u_in=0.05, sigma_band=1.0, eps_h=2.0, transition="smoothstep",
                 wall_model=True, wm_E=9.8, wm_kappa=0.41, wm_ysample=2.0, wm_tol=1e-4,
                 wm_maxit=10, force_form=0, modes=None, rotors=()):
        p = Params()
        p.nx, p.ny, p.nz, p.q = nx, ny, nz, q
        p.flow_axis = flow_axis
        p.open_boundaries = int(bool(open_boundaries))
        p.tau_mo, p.c_smag, p.u_in = tau_mo, c_smag, u_in
        p.sigma_band, p.eps_h = sigma_band, eps_h
        p.transition = 1 if transition == "linear" else 0
        p.wall_model = int(bool(wall_model))
        p.wm_E, p.wm_kappa, p.wm_ysample, p.wm_tol, p.wm_maxit = wm_E, wm_kappa, wm_ysample, wm_tol, wm_maxit
        p.force_form = int(force_form)
        self._modes = None
        if modes is not None and len(modes):
            self._modes = np.ascontiguousarray(modes, dtype=np.float64).reshape(-1, 9)
            p.n_modes = self._modes.shape[0]
            p.modes = _ptr(self._modes)
        else:
            p.n_modes = 0
        self._rotors = list(rotors)
        arr = (Rotor * max(1, len(self._rotors)))(*self._rotors)
        self._h = lib().or_create(C.byref(p), arr, len(self._rotors))
        if not self._h:
            raise ValueError("oracle: invalid parameters")
        self.shape = (nz, ny, nx)
        self.flow_axis = flow_axis
        self.q = q
        self.N = nx * ny * nz
        self.nrot = len(self._rotors)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().or_destroy(h)
            self._h = None

    @property
    def t(self) -> int:
        return lib().or_time(self._h)

    def step(self, n: int = 1):
        lib().or_step(self._h, int(n))

    def populations(self) -> np.ndarray:
        out = np.empty((self.q,) + self.shape)
        lib().or_get_populations(self._h, _ptr(out))
        return out

    def set_populations(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64).reshape((self.q,) + self.shape)
        lib().or_set_populations(self._h, _ptr(f))

    def init_equilibrium(self, rho, u):
        rho = np.ascontiguousarray(np.broadcast_to(rho, self.shape), dtype=np.float64)
        u = np.ascontiguousarray(np.broadcast_to(u, (3,) + self.shape), dtype=np.float64)
        lib().or_init_equilibrium(self._h, _ptr(rho), _ptr(u))

    def fields(self):
        rho = np.empty(self.shape)
        u = np.empty((3,) + self.shape)
        lib().or_fields(self._h, _ptr(rho), _ptr(u))
        return rho, u

    def forces(self):
        """(F, M, F_avg, M_avg), each (n_rotors, 3)."""
        n = max(1, self.nrot)
        F, M, Fa, Ma = (np.zeros((n, 3)) for _ in range(4))
        lib().or_forces(self._h, _ptr(F), _ptr(M), _ptr(Fa), _ptr(Ma))
        return F[:self.nrot], M[:self.nrot], Fa[:self.nrot], Ma[:self.nrot]

    def reset_average(self):
        lib().or_reset_average(self._h)

    def mass(self) -> float:
        return lib().or_mass(self._h)

    def geometry(self):
        phi = np.empty(self.shape, dtype=np.float32)
        d = np.empty(self.shape)
        fl = np.empty(self.shape, dtype=np.uint8)
        tag = np.empty(self.shape, dtype=np.int8)
        lib().or_geometry(self._h, _ptr(phi, _fp), _ptr(d), _ptr(fl, _u8p), _ptr(tag, _i8p))
        return phi, d, fl, tag

    def wall_state(self):
        du = np.empty(self.shape + (3,))
        S = np.empty(self.shape + (3, 3))
        ut = np.empty(self.shape)
        act = np.empty(self.shape, dtype=np.uint8)
        y1 = np.empty(self.shape + (3,))
        lib().or_wall_state(self._h, _ptr(du), _ptr(S), _ptr(ut), _ptr(act, _u8p), _ptr(y1))
        return du, S, ut, act, y1

    def inflow_plane(self, t: int) -> np.ndarray:
        dims = (self.shape[2], self.shape[1], self.shape[0])
        a = self.flow_axis
        nb, nc = dims[(a + 1) % 3], dims[(a + 2) % 3]
        out = np.empty((nc, nb, 3))
        lib().or_inflow_plane(self._h, int(t), _ptr(out))
        return out

    def set_d0(self, d0):
        """Static porosity multiplier d0 (shape (nz, ny, nx)); None restores d0 = 1."""
        if d0 is None:
            lib().or_set_d0(self._h, None)
            return
        self._d0 = np.ascontiguousarray(np.broadcast_to(d0, self.shape), dtype=np.float64)
        lib().or_set_d0(self._h, _ptr(self._d0))

    def set_pitch(self, k: int, pitch: float):
        if lib().or_set_pitch(self._h, int(k), float(pitch)):
            raise IndexError("rotor index")

    def freeze_sets(self, on: bool = True):
        """Hold the cell sets at the current pitches; porosity, normals and wall
        distances keep following set_pitch."""
        lib().or_freeze_sets(self._h, int(bool(on)))

    def adjoint(self, steps: int, avg_last: int, w_thrust, w_torque):
        """Run `steps` steps; return (J, dJ/dpitch[n_rotors], dJ/dd0 (nz, ny, nx)) for
        J = mean over the last avg_last steps of sum_k wT_k F_k.a_k + wQ_k M_k.a_k."""
        n = max(1, self.nrot)
        wT = np.zeros(n)
        wQ = np.zeros(n)
        wT[:self.nrot] = w_thrust
        wQ[:self.nrot] = w_torque
        J = np.zeros(1)
        gp = np.zeros(n)
        gd0 = np.zeros(self.shape)
        rc = lib().or_adjoint(self._h, int(steps), int(avg_last), _ptr(wT), _ptr(wQ), _ptr(J), _ptr(gp), _ptr(gd0))
        if rc:
            raise ValueError(f"oracle adjoint failed ({rc})")
        return float(J[0]), gp[:self.nrot], gd0

    def set_drive(self, k: int, inertia: float, k_gen: float = 0.0, q_gen0: float = 0.0):
        """Torque-driven rotation of rotor k from now on (I dOmega/dt = M.a - Q_gen)."""
        if lib().or_set_drive(self._h, int(k), float(inertia), float(k_gen), float(q_gen0)):
            raise ValueError("bad rotor index or inertia")

    def drive_state(self, k: int):
        """(theta, Omega) of rotor k at the current step."""
        th, om = C.c_double(), C.c_double()
        lib().or_drive_state(self._h, int(k), C.byref(th), C.byref(om))
        return th.value, om.value

    def fd_strain(self):
        """Central-difference rate of strain of the current velocity field, (nz, ny, nx, 3, 3)."""
        out = np.zeros(self.shape + (3, 3))
        lib().or_fd_strain(self._h, _ptr(out))
        return out

    def porosity_tangent(self):
        """d(d_rotor)/d(pitch) of the last porosity update, shape (nz, ny, nx)."""
        out = np.zeros(self.shape)
        lib().or_porosity_tangent(self._h, _ptr(out))
        return out

    def wall_tangent(self):
        """Run the porosity update and wall model of the current step (state not
        advanced) and return (d du/d pitch (nz,ny,nx,3), d S/d pitch (nz,ny,nx,3,3))."""
        ddu = np.zeros(self.shape + (3,))
        dS = np.zeros(self.shape + (3, 3))
        lib().or_wall_tangent(self._h, _ptr(ddu), _ptr(dS))
        return ddu, dS

    def newton_stats(self):
        it, ev = C.c_long(0), C.c_long(0)
        lib().or_newton_stats(self._h, C.byref(it), C.byref(ev))
        return it.value, ev.value


def from_workload(wl, rotor_kw=None, **overrides) -> Oracle:
    """Build an Oracle for a ``workloads.Workload``."""
    grids = wl.blade_grids()
    rotors = []
    for spec, g in zip(wl.rotors, grids):
        kw = dict(center=spec.center, axis=wl.flow_axis, omega=spec.omega(wl.u_in),
                  phase0=spec.phase0, pitch=spec.pitch, n_blades=spec.n_blades)
        if rotor_kw:
            kw.update(rotor_kw)
        rotors.append(make_rotor(g, **kw))
    kw = dict(q=wl.q, flow_axis=wl.flow_axis, tau_mo=wl.tau_mo, c_smag=wl.c_smag,
              u_in=wl.u_in, eps_h=wl.eps_h, modes=wl.modes(), rotors=rotors)
    kw.update(overrides)
    return Oracle(wl.nx, wl.ny, wl.nz, **kw)
