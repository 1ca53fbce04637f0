"""Grid-convergence analysis of the time-averaged thrust coefficient
(Sec. 4: Definition "Thrust coefficient", the experimental order of
convergence from a log-log regression, and Definition "Grid Convergence
Index").

The analysis functions are host arithmetic on a handful of numbers; the
study driver runs the rotor on the GPU library at several resolutions of the
synthetic rotor with the Reynolds number and the tip-speed ratio held fixed.
"""

from __future__ import annotations

import math

import numpy as np


def thrust_coefficient(thrust: float, radius: float, u_inf: float, rho: float = 1.0) -> float:
    """C_T = T / (1/2 rho pi r^2 U_inf^2) (Sec. 4, Definition "Thrust coefficient")."""
    return thrust / (0.5 * rho * math.pi * radius * radius * u_inf * u_inf)


def eoc(h, err) -> float:
    """Experimental order of convergence: slope of the least-squares line
    through (log h, log err) (Sec. 4, grid convergence analysis)."""
    h = np.asarray(h, dtype=np.float64)
    err = np.asarray(err, dtype=np.float64)
    slope, _ = np.polyfit(np.log(h), np.log(err), 1)
    return float(slope)


def apparent_order(f1: float, f2: float, f3: float, r: float) -> float:
    """Order p from three grids with a constant refinement ratio r (f1 finest):
    (f3 - f2) / (f2 - f1) = r^p for f(h) = f* + C h^p."""
    return math.log(abs((f3 - f2) / (f2 - f1))) / math.log(r)


def gci(f1: float, f2: float, r: float, p: float, fs: float = 1.25) -> float:
    """Grid Convergence Index of the fine-grid value f1 (Sec. 4, Definition
    "Grid Convergence Index"): F_s |(f2 - f1) / f1| / (r^p - 1), r = h2 / h1 > 1."""
    return fs * abs((f2 - f1) / f1) / (r ** p - 1.0)


def study_workload(radius: int, tsr: float = 6.0, u_in: float = 0.05, tau_ref: float = 0.5005,
                   radius_ref: int = 32, ladder: str = "reynolds"):
    """The synthetic rotor at resolution `radius` (cells per rotor radius):
    lattice 4R x 4R x 8R, rotor a quarter of the length downstream of the
    inlet, uniform inflow, tip-speed ratio `tsr` at every resolution.

    ladder "reynolds": the Reynolds number of the reference resolution at
    every R (nu scales with R: tau - 1/2 = (tau_ref - 1/2) R / R_ref), so the
    wall-normal spacing in wall units, and with it the first cell's y+,
    falls as the grid is refined.  ladder "yplus": the lattice viscosity of
    the reference (tau = tau_ref) at every R, so y+ of the first cell (its
    distance in cells times u_tau / nu) stays the same while the Reynolds
    number U R / nu grows with R: the refinement of a wall-modelled LES,
    which resolves the outer flow ever finer and models the same inner layer.
    ladder "interface": the y+ ladder with the porosity transition scaled with
    the rotor (eps_h = 2 R / R_ref cells, Definition "Lattice Porosity"), so
    the diffuse interface, and the wall set in its fluid half, cover the same
    fraction of the blade chord at every R."""
    from workloads.configs import Workload, _single
    n = 4 * radius
    eps_h = 2.0
    if ladder == "reynolds":
        tau = 0.5 + (tau_ref - 0.5) * radius / radius_ref
    elif ladder in ("yplus", "interface"):
        tau = tau_ref
        if ladder == "interface":
            eps_h = 2.0 * radius / radius_ref
    else:
        raise ValueError("ladder is 'reynolds', 'yplus' or 'interface'")
    # blade-grid padding: the fluid half of the transition, the sampling distance
    # and the trilinear corner stay inside the grid (and so inside the rotor box)
    margin = 4.0 if eps_h <= 2.0 else 0.5 * eps_h + 4.0
    return Workload(f"convergence_R{radius}_{ladder}", n, n, 2 * n, steps=0, tau_mo=tau, u_in=u_in, eps_h=eps_h,
                    grid_margin=margin, rotors=_single(n, n, 2 * n, float(radius), tsr))


def run_study(radii=(16, 32, 64, 128), revolutions_spinup: float = 3.0, revolutions_avg: float = 2.0,
              device=None, progress=None, wall_model: bool = True, ladder: str = "reynolds"):
    """C_T averaged over whole revolutions after a spin-up, at each resolution,
    on the GPU library.  Returns a dict with per-resolution results, the EOC
    against the finest grid and the GCI of the finest grid from the three
    finest (constant refinement ratio).  wall_model=False runs the porous
    blades without the wall function (resolved HLBM only)."""
    import torch
    from paper_2510_13726_b300 import Lattice
    rows = []
    for R in radii:
        wl = study_workload(R, ladder=ladder)
        om = wl.rotors[0].omega(wl.u_in)
        steps_rev = 2.0 * math.pi / om
        n_spin = int(round(revolutions_spinup * steps_rev))
        n_avg = int(round(revolutions_avg * steps_rev))
        lat = Lattice.from_workload(wl, device=device, wall_model=wall_model)
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(lat.stream)
        lat.step(n_spin)
        lat.forces(reset_avg=True)
        lat.step(n_avg)
        t1.record(lat.stream)
        t1.synchronize()
        _, Fa = lat.forces()
        T = float(Fa[0, wl.flow_axis])
        ms = t0.elapsed_time(t1)
        band = lat.rotor_band(0)
        wall = (band["flags"] & 2) > 0
        ut = band["utau"][wall]
        nu = (wl.tau_mo - 0.5) / 3.0
        rows.append({"R": R, "cells": wl.cells, "tau": wl.tau_mo, "eps_h": wl.eps_h, "Re": wl.u_in * R / nu,
                     "steps": n_spin + n_avg, "thrust": T, "C_T": thrust_coefficient(T, R, wl.u_in),
                     # wall units per lattice spacing, u_tau / nu, of the last step: median over the wall
                     # cells (a wall cell sits 0.5 to 1 spacing from the wall)
                     "yplus_per_cell_median": float(torch.median(ut / nu).item()) if ut.numel() else None,
                     "seconds": round(ms / 1e3, 2)})
        if progress:
            progress(rows[-1])
        lat.close()
        del lat
        torch.cuda.empty_cache()
    out = {"wall_model": bool(wall_model), "ladder": ladder, "resolutions": rows}
    ct = [r["C_T"] for r in rows]
    if len(rows) >= 3:
        h = [1.0 / r["R"] for r in rows[:-1]]
        err = [abs(c - ct[-1]) for c in ct[:-1]]
        if all(e > 0 for e in err):
            out["eoc"] = eoc(h, err)
        r = rows[-1]["R"] / rows[-2]["R"]
        p = apparent_order(ct[-1], ct[-2], ct[-3], r)
        out["apparent_order"] = p
        out["gci_finest"] = gci(ct[-1], ct[-2], r, p)
    return out


if __name__ == "__main__":
    import argparse
    import json
    import sys
    ap = argparse.ArgumentParser(description="grid-convergence study of the synthetic rotor on one GPU")
    ap.add_argument("--radii", default="16,32,64,128")
    ap.add_argument("--spinup", type=float, default=3.0, help="revolutions before averaging")
    ap.add_argument("--average", type=float, default=2.0, help="revolutions averaged")
    ap.add_argument("--no-wall-model", action="store_true", help="porous blades without the wall function")
    ap.add_argument("--ladder", default="reynolds", choices=["reynolds", "yplus", "interface"],
                    help="hold the Reynolds number (reynolds), the first cell's y+ (yplus), or y+ and the "
                         "porosity transition relative to the rotor (interface) across R")
    args = ap.parse_args()
    radii = tuple(int(v) for v in args.radii.split(","))
    res = run_study(radii, args.spinup, args.average, wall_model=not args.no_wall_model, ladder=args.ladder,
                    progress=lambda row: print(json.dumps(row), file=sys.stderr, flush=True))
    print(json.dumps(res))
