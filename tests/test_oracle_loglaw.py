"""Pins of the oracle's whole-cell wall model in the log-law regime (Sec. 2.2.1;
no GPU).

The wall model of a wall cell x (Sec. 2.2.1, Eqs. (u+), (y+), (spalding),
(implicitWF), (guess), and the velocity feedback "added to the velocity moment
of the porous medium") takes the fluid velocity at the sampling point
x + y_s n, removes the wall's own velocity and the wall-normal part, solves the
wall function for u_tau at the sample's wall distance |y_1| + y_s, and returns
the modelled velocity u_tau u+(y_1+) along the tangential direction together
with the strain of the straight velocity profile between the wall cell and the
sample.  These tests build velocity fields whose values at the sample point
are known in closed form (a pure log law u = u_tau/kappa ln(E y u_tau/nu)
around a flat wall at an oblique angle, with a normal component and a moving
wall added) and compare every output of the oracle with values computed here
from the definitions alone:

  * the sample velocity by a library trilinear interpolation
    (scipy.ndimage.map_coordinates, order 1) of the prescribed cell field,
  * u_tau and u+ as roots of the explicit Eq. (spalding) by bracketing
    (scipy.optimize.brentq), not by the oracle's Newton,
  * the strain as the symmetric gradient, by central differences, of the
    straight shear profile through the wall cell and the sample point,
  * the log law ln(E y+)/kappa, which the wall function approaches with the
    exact gap ln(1 + (P(kappa u+) - E u+)/(E y+))/kappa, where P is the cubic
    Taylor polynomial of exp that Eq. (spalding) subtracts.

Each of these mistakes in the assembly fails at least one test below: u+
taken at the sample's wall distance instead of y_1+; the sample's wall
distance taken as y_s instead of |y_1| + y_s; a factor 2 in the strain; the
normal part of the relative velocity kept; the wall velocity not subtracted;
a cell newly in the wall set warm-started (or the cold start of Eq. (guess)
taken at another distance).
"""

import math

import numpy as np
import pytest
from scipy.ndimage import map_coordinates
from scipy.optimize import brentq

import oracle as O
from workloads import BladeGrid

E, KAPPA = 9.8, 0.41
TAU = 0.50005
NU = (TAU - 0.5) / 3.0
YS = 2.0                                  # sampling distance (cells), the default


def _yplus(up):
    """Eq. (spalding): y+ as an explicit function of u+."""
    k = KAPPA * up
    return up + (math.exp(k) - 1.0 - k - k * k / 2.0 - k ** 3 / 6.0) / E


def _uplus(yp):
    return brentq(lambda v: _yplus(v) - yp, 1e-9, 80.0, xtol=1e-15, rtol=1e-15)


def _utau(u, y):
    """Root of Eq. (implicitWF) in u_tau for tangential speed u at wall distance y."""
    return brentq(lambda ut: _yplus(u / ut) - y * ut / NU, u / 150.0, u, xtol=1e-16, rtol=1e-15)


def _loglaw_gap(up, yp):
    """Exact u+ - ln(E y+)/kappa on the Spalding curve (rewrite of Eq. (spalding))."""
    k = KAPPA * up
    P = 1.0 + k + k * k / 2.0 + k ** 3 / 6.0
    return math.log1p((P - E * up) / (E * yp)) / KAPPA


def _plane_grid(shape, center, n_hat, p0, h=0.5):
    """Rotor-frame level set of the plane n.(x - p0) = 0 (solid on the side
    n.(x - p0) < 0) for a rotor about z at angle 0 and pitch 0, whose blade
    frame (R, T, A) is the lab frame shifted by the rotor centre."""
    nx, ny, nz = shape
    lo = [-center[0] - 2, -center[1] - 2, -center[2] - 2]
    hi = [nx + 1 - center[0], ny + 1 - center[1], nz + 1 - center[2]]
    g = [int(round((hi[k] - lo[k]) / h)) + 1 for k in range(3)]
    R = lo[0] + h * np.arange(g[0])
    T = lo[1] + h * np.arange(g[1])
    A = lo[2] + h * np.arange(g[2])
    AA, TT, RR = np.meshgrid(A, T, R, indexing="ij")
    phi = (n_hat[0] * (RR + center[0] - p0[0]) + n_hat[1] * (TT + center[1] - p0[1])
           + n_hat[2] * (AA + center[2] - p0[2]))
    return BladeGrid(sdf=np.ascontiguousarray(phi.astype(np.float32)), origin=tuple(lo), spacing=h,
                     radius=1.0, hub_radius=0.0, chord_root=1.0, chord_tip=1.0)


def _log_profile(y, ut):
    return ut / KAPPA * np.log(E * np.maximum(y, 1e-3) * ut / NU)


SHAPE = (20, 20, 8)
N_HAT = np.array([0.35, 1.0, 0.25]) / np.linalg.norm([0.35, 1.0, 0.25])
P0 = np.array([9.6, 6.3, 3.7])
UT_STAR = 0.002


def _setup(omega=0.0, center=(9.5, 9.5, 3.5), u_normal=0.0, n_hat=N_HAT, p0=P0, **kw):
    """Oracle on a periodic box with the plane n.(x - p0) = 0 as its only
    rotor and the velocity field u = u_wall(x) + U_log(phi) t + u_normal n
    (U_log = the log law of UT_STAR at the exact distance phi from the plane,
    0 in the solid; t a fixed tangential direction); returns the oracle, the
    exact distance field and the velocity field (3, nz, ny, nx)."""
    nx, ny, nz = SHAPE
    n_hat = np.asarray(n_hat, float)
    t0 = _tangent(n_hat)
    grid = _plane_grid(SHAPE, center, n_hat, p0)
    rot = O.make_rotor(grid, center=center, axis=2, omega=omega, n_blades=1, hub_radius=0.0)
    o = O.Oracle(nx, ny, nz, open_boundaries=False, tau_mo=TAU, c_smag=0.1, u_in=0.0, wall_model=True,
                 rotors=[rot], **kw)
    Z, Y, X = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    phi = n_hat[0] * (X - p0[0]) + n_hat[1] * (Y - p0[1]) + n_hat[2] * (Z - p0[2])
    uw = _solid_velocity(omega, center, X, Y, Z)
    U = np.where(phi > 0.05, _log_profile(phi, UT_STAR), 0.0)
    u = uw + U[None] * t0[:, None, None, None] + u_normal * n_hat[:, None, None, None]
    o.init_equilibrium(np.ones(o.shape), u)
    return o, phi, u


def _tangent(n_hat):
    t = np.cross(n_hat, [0.0, 0.0, 1.0])
    if np.linalg.norm(t) < 1e-6:
        t = np.cross(n_hat, [1.0, 0.0, 0.0])
    return t / np.linalg.norm(t)


def _solid_velocity(omega, c, X, Y, Z):
    """Rigid rotation about +z through c: Omega z x (x - c)."""
    X = np.asarray(X, float)
    return np.stack([-omega * (np.asarray(Y, float) - c[1]), omega * (X - c[0]), 0.0 * X])


def _interior_wall_cells(phi):
    """Wall cells (0 <= phi < eps_h/2 = 1) whose sampling point's eight
    trilinear corners lie inside the box (no periodic wrap of the plane)."""
    nx, ny, nz = SHAPE
    cells = []
    for z, y, x in zip(*np.nonzero((phi >= 0.0) & (phi < 1.0))):
        xs = np.array([x, y, z]) + YS * N_HAT
        lo = np.floor(xs)
        if np.all(lo >= 0) and np.all(lo + 1 <= np.array([nx, ny, nz]) - 1):
            cells.append((int(x), int(y), int(z)))
    assert len(cells) > 40
    return cells


def _expected(u, phi, cells, omega=0.0, center=(9.5, 9.5, 3.5)):
    """Closed-form wall-model outputs for each cell: (|u_t|, t_hat, y1, u_tau, du, S)."""
    out = []
    for x, y, z in cells:
        xs = np.array([x, y, z], float) + YS * N_HAT
        coords = np.array([[xs[2]], [xs[1]], [xs[0]]])
        us = np.array([map_coordinates(u[k], coords, order=1, mode="grid-wrap")[0] for k in range(3)])
        rel = us - _solid_velocity(omega, center, x, y, z)
        ut_vec = rel - rel.dot(N_HAT) * N_HAT
        utm = np.linalg.norm(ut_vec)
        t_hat = ut_vec / utm
        y1 = max(phi[z, y, x], 0.5)
        utau = _utau(utm, y1 + YS)
        uw = utau * _uplus(y1 * utau / NU)

        def shear(p):
            # straight profile along n through (y1, uw) and (y1 + y_s, |u_t|)
            s = N_HAT.dot(p - np.array([x, y, z], float))
            return t_hat * (uw + (utm - uw) * (s - 0.0) / YS)

        G = np.zeros((3, 3))
        for b in range(3):
            e = np.zeros(3)
            e[b] = 0.5
            G[:, b] = (shear(np.array([x, y, z], float) + e) - shear(np.array([x, y, z], float) - e))
        out.append((utm, t_hat, y1, utau, uw * t_hat, 0.5 * (G + G.T)))
    return out


@pytest.mark.parametrize("case", ["static", "normal_flow", "moving_wall"])
def test_wall_model_closed_form_on_oblique_wall(case):
    """One evaluation of the wall model (tolerance 1e-13, up to 100 Newton
    iterations, so the solve reaches its root) on the log-law field: u_tau,
    the modelled velocity and the strain of every interior wall cell equal the
    closed form to the binary32 rounding of the level set (1e-5 relative)."""
    kw = {"static": {}, "normal_flow": {"u_normal": 0.012},
          "moving_wall": {"omega": 6e-5, "center": (-150.0, -120.0, 3.5)}}[case]
    om, ctr = kw.get("omega", 0.0), kw.get("center", (9.5, 9.5, 3.5))
    o, phi, u = _setup(wm_tol=1e-13, wm_maxit=100, **kw)
    cells = _interior_wall_cells(phi)
    o.step(1)
    du, S, ut, act, y1v = o.wall_state()
    _, _, fl, _ = o.geometry()
    for (x, y, z), (utm, t_hat, y1, utau, du_ref, S_ref) in zip(cells, _expected(u, phi, cells, om, ctr)):
        assert fl[z, y, x] & 2 and act[z, y, x] == 1
        assert abs(np.linalg.norm(y1v[z, y, x]) - y1) < 2e-5
        assert abs(ut[z, y, x] / utau - 1) < 1e-5
        assert np.abs(du[z, y, x] - du_ref).max() < 1e-5 * np.linalg.norm(du_ref)
        g = (utm - np.linalg.norm(du_ref)) / YS
        assert np.abs(S[z, y, x] - S_ref).max() < 1e-5 * abs(g)
        # a simple shear: traceless, |S| = sqrt(2 S:S) = |g|, S n = g t / 2
        assert abs(np.trace(S[z, y, x])) < 1e-12
        assert abs(math.sqrt(2 * np.sum(S[z, y, x] ** 2)) / abs(g) - 1) < 1e-5
        assert np.abs(S[z, y, x] @ N_HAT - 0.5 * g * t_hat).max() < 1e-5 * abs(g)


@pytest.mark.parametrize("n_hat,p0", [((0.0, 1.0, 0.0), (0.0, 3.3, 0.0)), ((-1.0, 0.0, 0.0), (15.7, 0.0, 0.0))])
def test_wall_model_follows_the_log_law(n_hat, p0):
    """A lattice-aligned wall 0.7 cells from the wall cells, so that every
    sampling point is a lattice node and sits at the exact wall distance
    |y1| + y_s = 2.7 (no interpolation): the solved friction velocity differs
    from the log-law field's UT_STAR only by the wall function's own gap to the
    log law at the sample (y+ = 324: u_tau 0.23 % above, solved here exactly), and the
    modelled velocity is u_tau (ln(E y1+)/kappa + gap) with the exact gap of
    Eq. (spalding) at y1+ ~ 84 (1.6 % below the log law, checked within 2 %)."""
    o, phi, u = _setup(n_hat=n_hat, p0=np.array(p0), wm_tol=1e-13, wm_maxit=100)
    sel = (phi > 0.69) & (phi < 0.71)
    assert sel.sum() == SHAPE[2] * (SHAPE[0] if n_hat[1] else SHAPE[1])
    o.step(1)
    du, _, ut, act, _ = o.wall_state()
    ys = 0.7 + YS
    u_samp = UT_STAR / KAPPA * math.log(E * ys * UT_STAR / NU)
    ut_ref = _utau(u_samp, ys)
    assert 0.0 < ut_ref / UT_STAR - 1 < 3e-3      # Spalding's u+ lies below the log law
    for z, y, x in zip(*np.nonzero(sel)):
        assert act[z, y, x] == 1
        utau = ut[z, y, x]
        assert abs(utau / ut_ref - 1) < 1e-6
        y1p = 0.7 * utau / NU
        assert y1p > 80.0                          # first cell in the log region
        up = np.linalg.norm(du[z, y, x]) / utau
        log_up = math.log(E * y1p) / KAPPA
        assert abs(up - (log_up + _loglaw_gap(up, y1p))) < 1e-6 * up
        assert abs(up / log_up - 1) < 0.02
        assert np.abs(du[z, y, x] / np.linalg.norm(du[z, y, x]) - _tangent(np.array(n_hat))).max() < 1e-12


def test_newton_start_values_of_eq_guess():
    """Eq. (guess) with one Newton iteration per evaluation (tolerance 0, so
    exactly one step is taken): a cell entering the wall set starts from
    sqrt(nu |u_t| / y_s) and the next evaluation, the cell having been active,
    starts from the previous u_tau.  The expected iterates are computed here
    with the derivative of Eq. (implicitWF) by complex-step differentiation."""
    o, phi, u = _setup(wm_tol=0.0, wm_maxit=1)
    f0 = o.populations()
    cells = _interior_wall_cells(phi)
    exp = _expected(u, phi, cells)

    def f(ut, um, y):
        v = um / ut
        k = KAPPA * v
        return v + (np.exp(k) - 1.0 - k - k * k / 2.0 - k ** 3 / 6.0) / E - y * ut / NU

    def newton(ut, um, y):
        d = f(complex(ut, 1e-30), um, y).imag / 1e-30
        return ut - f(ut, um, y) / d

    o.step(1)
    _, _, ut1, act, _ = o.wall_state()
    o.set_populations(f0)               # same populations: only the start value differs
    o.step(1)
    _, _, ut2, _, _ = o.wall_state()
    for (x, y, z), (utm, _, y1, utau, _, _) in zip(cells, exp):
        g0 = math.sqrt(NU * utm / YS)
        it1 = newton(g0, utm, y1 + YS)
        assert it1 > 0
        assert abs(ut1[z, y, x] / it1 - 1) < 1e-6
        it2 = newton(it1, utm, y1 + YS)
        assert abs(ut2[z, y, x] / it2 - 1) < 1e-6
        assert abs(it2 - utau) < abs(it1 - utau)     # the warm start moves towards the root


def _log_channel(wall_model):
    """Periodic channel between two lattice-aligned porous walls (solid for
    y < 3.3 and y > 35.7, flow along x), initialised with the log law of
    UT_STAR from each wall (centreline y+ ~ 1900), run for 1000 steps."""
    nx, ny, nz = 4, 40, 4
    a, b = 3.3, 35.7
    c, h = (1.5, 19.5, 1.5), 0.5
    lo = [-c[0] - 2, -c[1] - 2, -c[2] - 2]
    hi = [nx + 1 - c[0], ny + 1 - c[1], nz + 1 - c[2]]
    g = [int(round((hi[k] - lo[k]) / h)) + 1 for k in range(3)]
    A = lo[2] + h * np.arange(g[2])
    T = lo[1] + h * np.arange(g[1])
    R = lo[0] + h * np.arange(g[0])
    _, TT, _ = np.meshgrid(A, T, R, indexing="ij")
    y = TT + c[1]
    grid = BladeGrid(sdf=np.ascontiguousarray(np.minimum(y - a, b - y).astype(np.float32)), origin=tuple(lo),
                     spacing=h, radius=1.0, hub_radius=0.0, chord_root=1.0, chord_tip=1.0)
    rot = O.make_rotor(grid, center=c, axis=2, omega=0.0, n_blades=1, hub_radius=0.0)
    o = O.Oracle(nx, ny, nz, open_boundaries=False, tau_mo=TAU, c_smag=0.1, u_in=0.0, wall_model=wall_model,
                 rotors=[rot])
    ys = np.arange(ny)
    phi = np.minimum(ys - a, b - ys)
    U = np.where(phi > 0.05, _log_profile(phi, UT_STAR), 0.0)
    u = np.zeros((3, nz, ny, nx))
    u[0] = U[None, :, None]
    o.init_equilibrium(np.ones((nz, ny, nx)), u)
    o.step(1000)
    _, uu = o.fields()
    return o, phi, U, uu


def test_log_law_channel_is_kept_by_the_wall_model():
    """Wall-modelled channel at y1+ ~ 84 (first cell 0.7 from the wall): the
    log-law profile is the near-wall state the wall function encodes, so the
    scheme keeps it.  Over 1000 steps (the flow, unforced, loses u_tau^2/h of
    its mean speed per step: 0.5 % at the centreline) the cells from the
    sampling distance on stay on ln(E y+)/kappa within 1 %, the solved u_tau
    returns to the log law's (within 0.5 % of the exact solve at the
    sample), both walls alike; the wall cell and its neighbour, inside the
    2-cell diffuse interface, keep 85 % and 90 % of the log-law value.
    Without the wall model the same channel's first cell loses more than 90 %
    and its neighbour more than 40 % (a resolved no-slip wall at this
    spacing), so the near-wall profile is the wall model's doing."""
    o, phi, U, uu = _log_channel(True)
    prof = uu[0, 1, :, 1]
    assert np.abs(uu[0] - prof[None, :, None]).max() < 1e-12          # uniform along x and z
    assert np.abs(uu[1:]).max() < 1e-9 * prof.max()
    far = (phi >= 2.69) & (phi <= 16.3)
    assert np.abs(prof[far] / U[far] - 1).max() < 0.01
    _, _, ut, act, _ = o.wall_state()
    ys = 0.7 + YS
    ut_ref = _utau(UT_STAR / KAPPA * math.log(E * ys * UT_STAR / NU), ys)
    wall = np.nonzero(np.abs(phi - 0.7) < 1e-9)[0]
    assert list(wall) == [4, 35]
    for j in wall:
        assert act[1, j, 1] == 1 and abs(ut[1, j, 1] / ut_ref - 1) < 5e-3
    assert abs(ut[1, 4, 1] / ut[1, 35, 1] - 1) < 1e-9
    for j, keep in ((4, 0.85), (5, 0.90), (35, 0.85), (34, 0.90)):
        assert prof[j] / U[j] > keep
    _, _, _, off = _log_channel(False)
    p_off = off[0, 1, :, 1]
    assert p_off[4] / U[4] < 0.1 and p_off[5] / U[5] < 0.6
