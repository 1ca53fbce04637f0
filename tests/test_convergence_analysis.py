"""Pins of the grid-convergence analysis (Sec. 4): on a manufactured
sequence f(h) = f* + C h^p the regression slope and the three-grid order
recover p exactly, and the Grid Convergence Index divided by its safety
factor is exactly the relative error of the fine-grid value; the thrust
coefficient is the thrust of the reference dynamic pressure on the rotor
disk; the study workloads hold Reynolds number and tip-speed ratio."""

import math

import numpy as np
import pytest

from paper_2510_13726_b300 import convergence as C


@pytest.mark.parametrize("p", [1.0, 1.38, 2.1])
def test_orders_recovered_on_manufactured_sequence(p):
    fstar, c = 0.963, -0.7
    h = np.array([1 / 5, 1 / 10, 1 / 20, 1 / 40])
    f = fstar + c * h ** p
    assert abs(C.eoc(h, np.abs(f - fstar)) - p) < 1e-12
    assert abs(C.apparent_order(f[3], f[2], f[1], 2.0) - p) < 1e-10


@pytest.mark.parametrize("p,r", [(1.38, 2.0), (2.1, 1.5), (2.0, 3.0)])
def test_gci_is_the_fine_grid_error(p, r):
    fstar, c, h1 = 0.963, 0.4, 0.01
    f1 = fstar + c * h1 ** p
    f2 = fstar + c * (r * h1) ** p
    g = C.gci(f1, f2, r, p, fs=1.25)
    assert abs(g / 1.25 - abs(f1 - fstar) / abs(f1)) < 1e-12


def test_thrust_coefficient_of_the_dynamic_pressure_on_the_disk():
    R, U, rho = 64.0, 0.05, 1.0
    assert abs(C.thrust_coefficient(0.5 * rho * math.pi * R * R * U * U, R, U, rho) - 1.0) < 1e-15
    # invariant under a change of length scale at fixed velocity: T ~ R^2
    assert abs(C.thrust_coefficient(4 * 1.3, 2 * R, U) - C.thrust_coefficient(1.3, R, U)) < 1e-15


def test_study_workloads_hold_reynolds_number_and_tip_speed_ratio():
    ws = [C.study_workload(R) for R in (16, 32, 64, 128)]
    re = [w.u_in * 2 * w.rotors[0].radius / ((w.tau_mo - 0.5) / 3) for w in ws]
    tsr = [w.rotors[0].omega(w.u_in) * w.rotors[0].radius / w.u_in for w in ws]
    assert max(re) - min(re) < 1e-9 * re[0]
    assert max(tsr) - min(tsr) < 1e-12
    assert ws[1].tau_mo == 0.5005
    for w in ws:
        assert (w.nx, w.ny, w.nz) == (4 * w.rotors[0].radius, 4 * w.rotors[0].radius, 8 * w.rotors[0].radius)
