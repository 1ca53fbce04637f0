"""Synthetic three-bladed NACA 4412 rotor: one blade voxelised on a grid.

The paper voxelises each moving element in its own reference grid at twice
the fluid resolution and embeds that grid into the lattice porosity every
step (Sec. 3.1).  The paper's rotor geometry (an STL file) is not available,
so a synthetic rotor stands in:

* NACA 4412 sections (public 4-digit formula, closed trailing edge),
* chord varying linearly from ``chord_root`` at the hub to ``chord_tip`` at
  the tip, twist varying linearly from ``twist_root`` to ``twist_tip``
  (degrees), sections placed about their quarter-chord point,
* a hub sphere (handled analytically by the consumers, not voxelised here).

The grid holds ONE blade in the blade frame (R, T, A):

* R  -- span direction (radial, through the rotor centre),
* T  -- tangential direction (direction of positive rotation),
* A  -- rotor axis (downstream).

The leading edge points to +T and the suction side to +A, so a rotor turning
with positive angular velocity about +A in a flow along +A extracts power.
The signed distance is negative inside the blade.  The blade SDF is the
maximum of the scaled section distance and the two radial caps, which is an
approximate distance; it is input data and both sides sample the same
float32 values.  Blade pitch and azimuth are applied by the consumers as
rigid rotations of the query point, so they are not baked in here.
"""

from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass
class BladeGrid:
    """One blade's signed-distance grid.

    ``sdf[k, j, i]`` is the value at blade-frame point
    ``origin + spacing * (i, j, k)`` with i along R, j along T, k along A.
    """

    sdf: np.ndarray            # float32, shape (gz, gy, gx), C-contiguous
    origin: tuple              # (R0, T0, A0) in lattice cells
    spacing: float             # node spacing in lattice cells (0.5)
    radius: float              # tip radius R
    hub_radius: float          # hub sphere radius
    chord_root: float
    chord_tip: float

    @property
    def shape(self):
        return self.sdf.shape


def naca4_polygon(m: float = 0.04, p: float = 0.4, t: float = 0.12, n: int = 161):
    """Closed NACA 4-digit profile polygon in chord units (LE at 0, TE at 1).

    Upper surface runs TE->LE, lower surface LE->TE; the first and last
    points coincide at the closed trailing edge.
    """
    beta = np.linspace(0.0, np.pi, n)
    xc = 0.5 * (1.0 - np.cos(beta))
    yt = 5.0 * t * (0.2969 * np.sqrt(xc) - 0.1260 * xc - 0.3516 * xc**2
                    + 0.2843 * xc**3 - 0.1036 * xc**4)
    front = xc < p
    yc = np.where(front, m / p**2 * (2 * p * xc - xc**2),
                  m / (1 - p) ** 2 * ((1 - 2 * p) + 2 * p * xc - xc**2))
    dyc = np.where(front, 2 * m / p**2 * (p - xc), 2 * m / (1 - p) ** 2 * (p - xc))
    th = np.arctan(dyc)
    xu, yu = xc - yt * np.sin(th), yc + yt * np.cos(th)
    xl, yl = xc + yt * np.sin(th), yc - yt * np.cos(th)
    px = np.concatenate([xu[::-1], xl[1:]])
    py = np.concatenate([yu[::-1], yl[1:]])
    px[-1], py[-1] = px[0], py[0]
    return px, py


def _polygon_sdf(px, py, qx, qy, chunk=1 << 15):
    """Signed distance from points (qx, qy) to a closed polygon, negative inside."""
    ax, ay = px[:-1], py[:-1]
    bx, by = px[1:], py[1:]
    ex, ey = bx - ax, by - ay
    ee = ex * ex + ey * ey
    out = np.empty(qx.shape, dtype=np.float64)
    fx, fy = qx.ravel(), qy.ravel()
    of = out.ravel()
    for s in range(0, fx.size, chunk):
        x = fx[s:s + chunk, None]
        y = fy[s:s + chunk, None]
        wx, wy = x - ax, y - ay
        h = np.clip((wx * ex + wy * ey) / ee, 0.0, 1.0)
        dx, dy = wx - h * ex, wy - h * ey
        dist = np.sqrt(np.min(dx * dx + dy * dy, axis=1))
        # even-odd crossing count of a ray towards +x
        cond = (ay <= y) != (by <= y)
        xint = ax + (y - ay) * ex / np.where(ey == 0.0, 1.0, ey)
        inside = np.sum(cond & (x < xint), axis=1) % 2 == 1
        of[s:s + chunk] = np.where(inside, -dist, dist)
    return out


class _SectionTable:
    """Bilinear table of the unit-chord NACA 4412 section signed distance."""

    def __init__(self, res: int = 160):
        self.x0, self.x1 = -0.6, 1.6
        self.y0, self.y1 = -0.6, 0.6
        self.h = 1.0 / res
        nx = int(round((self.x1 - self.x0) / self.h)) + 1
        ny = int(round((self.y1 - self.y0) / self.h)) + 1
        xs = self.x0 + self.h * np.arange(nx)
        ys = self.y0 + self.h * np.arange(ny)
        X, Y = np.meshgrid(xs, ys)
        px, py = naca4_polygon()
        self.table = _polygon_sdf(px, py, X, Y).reshape(ny, nx)

    def __call__(self, xi, eta):
        nyt, nxt = self.table.shape
        gx = (xi - self.x0) / self.h
        gy = (eta - self.y0) / self.h
        inside = (gx >= 0) & (gx <= nxt - 1.000001) & (gy >= 0) & (gy <= nyt - 1.000001)
        gxc = np.clip(gx, 0, nxt - 1.000001)
        gyc = np.clip(gy, 0, nyt - 1.000001)
        i0 = np.floor(gxc).astype(np.int64)
        j0 = np.floor(gyc).astype(np.int64)
        tx, ty = gxc - i0, gyc - j0
        T = self.table
        v = ((1 - tx) * (1 - ty) * T[j0, i0] + tx * (1 - ty) * T[j0, i0 + 1]
             + (1 - tx) * ty * T[j0 + 1, i0] + tx * ty * T[j0 + 1, i0 + 1])
        # far field: distance to the chord segment minus half the thickness
        far = np.hypot(xi - np.clip(xi, 0.0, 1.0), eta) - 0.06
        return np.where(inside, v, np.maximum(far, 0.5))


_TABLE = None


def _section_table():
    global _TABLE
    if _TABLE is None:
        _TABLE = _SectionTable()
    return _TABLE


def make_blade_grid(radius: float = 12.0, hub_radius: float | None = None,
                    chord_root: float | None = None, chord_tip: float | None = None,
                    twist_root: float = 20.0, twist_tip: float = 2.0,
                    spacing: float = 0.5, margin: float = 4.0) -> BladeGrid:
    """Voxelise one blade of the synthetic rotor.

    Defaults follow the 12-cell rotor (hub radius 2, chord 3 -> 1.5 cells);
    every length scales with ``radius / 12`` when not given.
    """
    s = radius / 12.0
    hub = 2.0 * s if hub_radius is None else hub_radius
    c_root = 3.0 * s if chord_root is None else chord_root
    c_tip = 1.5 * s if chord_tip is None else chord_tip
    r_root = 0.5 * hub                     # blade root buried inside the hub sphere
    w = 0.85 * max(c_root, c_tip) + margin
    R0, R1 = r_root - margin, radius + margin
    gx = int(np.ceil((R1 - R0) / spacing)) + 1
    gy = gz = int(np.ceil(2 * w / spacing)) + 1
    origin = (R0, -0.5 * (gy - 1) * spacing, -0.5 * (gz - 1) * spacing)
    r = origin[0] + spacing * np.arange(gx)
    T = origin[1] + spacing * np.arange(gy)
    A = origin[2] + spacing * np.arange(gz)
    tab = _section_table()
    frac = np.clip((r - hub) / (radius - hub), 0.0, 1.0)
    chord = c_root + (c_tip - c_root) * frac
    beta = np.deg2rad(twist_root + (twist_tip - twist_root) * frac)
    sdf = np.empty((gz, gy, gx), dtype=np.float32)
    Tg, Ag = np.meshgrid(T, A)           # shape (gz, gy)
    for i in range(gx):
        c, b = chord[i], beta[i]
        # chord direction (LE -> TE) and suction-side normal in the (T, A) plane
        xi = (Tg * -np.cos(b) + Ag * np.sin(b)) / c + 0.25
        eta = (Tg * np.sin(b) + Ag * np.cos(b)) / c
        d2 = c * tab(xi, eta)
        caps = max(r[i] - radius, r_root - r[i])
        sdf[:, :, i] = np.maximum(d2, caps).astype(np.float32)
    return BladeGrid(sdf=np.ascontiguousarray(sdf), origin=tuple(float(v) for v in origin),
                     spacing=float(spacing), radius=float(radius), hub_radius=float(hub),
                     chord_root=float(c_root), chord_tip=float(c_tip))


def blade_box_extent(grid: BladeGrid, extra: float = 2.0):
    """Conservative (in-plane radius, axial half-length) outside which every
    blade-grid sample is out of range and the hub sphere is farther than
    ``extra`` cells, for any rotor angle and any pitch."""
    gz, gy, gx = grid.sdf.shape
    h = grid.spacing
    R0, T0, A0 = grid.origin
    rmax = max(abs(R0), abs(R0 + h * (gx - 1)))
    tmax = max(abs(T0), abs(T0 + h * (gy - 1)))
    amax = max(abs(A0), abs(A0 + h * (gz - 1)))
    w = float(np.hypot(tmax, amax))          # pitch mixes T and A
    in_plane = max(float(np.hypot(rmax, w)), grid.hub_radius + extra)
    axial = max(w, grid.hub_radius + extra)
    return in_plane + 1.0, axial + 1.0
