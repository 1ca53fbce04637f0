"""Pins of the oracle's wall function and Newton solvers (Sec. 2.2.1; no GPU)."""

import inspect
import math

import pytest

import oracle as O


def test_paper_constants_are_the_defaults(golden):
    sig = inspect.signature(O.Oracle.__init__).parameters
    assert sig["wm_E"].default == golden["wall_function_E"]["value"]
    assert sig["wm_kappa"].default == golden["wall_function_kappa"]["value"]
    assert sig["wm_tol"].default == golden["newton_tolerance"]["value"]
    assert sig["wm_maxit"].default == golden["newton_max_iterations"]["value"]
    assert sig["u_in"].default == golden["lattice_velocity"]["value"]


def test_viscous_sublayer_limit():
    """For y+ -> 0 the wall function reduces to the linear sublayer u+ = y+;
    because Eq. (spalding) subtracts the exponential's Taylor terms up to the
    cubic, the deviation is of fourth order, (kappa y+)^4 / (24 E)."""
    for yp in (1e-3, 1e-2, 0.1, 0.5, 1.0):
        up = O.spalding_uplus(yp, tol=1e-14, maxit=60)
        lead = (0.41 * yp) ** 4 / (24 * 9.8)
        assert up <= yp
        assert abs((yp - up) - lead) <= 0.3 * lead + 1e-14


@pytest.mark.parametrize("yp", [1e3, 3e3, 1e4, 3e4])
def test_log_law_limit(yp):
    """For large y+ the Spalding law approaches the log law u+ = ln(E y+)/kappa."""
    up = O.spalding_uplus(yp, tol=1e-14, maxit=60)
    assert abs(up - math.log(9.8 * yp) / 0.41) < 0.05


@pytest.mark.parametrize("up", [0.3, 2.0, 5.0, 11.0, 18.0, 25.0])
def test_spalding_round_trip(up):
    """u+ -> y+ by Eq. (spalding), then the inverse solve recovers u+."""
    yp = O.spalding_yplus(up)
    assert yp >= up                       # the correction term is non-negative
    back = O.spalding_uplus(yp, tol=1e-14, maxit=60)
    assert abs(back - up) < 1e-9 * max(1.0, up)


@pytest.mark.parametrize("up", [3.0, 8.0, 14.0, 21.0])
@pytest.mark.parametrize("ut", [2e-3, 1e-2, 4e-2])
def test_newton_recovers_friction_velocity(up, ut):
    """Build a consistent (u, y) from a chosen u_tau via Eqs. (u+), (y+),
    (spalding); the Newton iteration on Eq. (implicitWF) from the initial
    guess of Eq. (guess) returns that u_tau."""
    nu = (0.5005 - 0.5) / 3.0
    yp = O.spalding_yplus(up)
    y = yp * nu / ut
    u = up * ut
    guess = math.sqrt(nu * u / y)
    tight, _ = O.wall_newton(u, y, nu, guess, tol=1e-15, maxit=100)
    assert abs(tight - ut) < 1e-10 * ut
    # with the paper's stopping rule (|df| < 1e-4, at most 10 iterations) a
    # cold start far in the log region needs the warm start of the following
    # steps (Eq. (guess), first case); a few warm-started calls converge
    r = guess
    for call in range(6):
        r, it = O.wall_newton(u, y, nu, r)
        assert it <= 10 and r > 0
    assert abs(r - ut) < 2e-3 * ut


def test_newton_warm_start_and_guard():
    """A warm start at the previous solution converges at once; a start so
    large that the Newton step would turn negative is halved instead, so the
    iterate stays positive."""
    nu = 1e-4
    ut, up = 0.02, 12.0
    yp = O.spalding_yplus(up)
    y, u = yp * nu / ut, up * ut
    r, it = O.wall_newton(u, y, nu, ut)
    assert it == 1 and abs(r - ut) < 1e-9
    for start in (3 * ut, 50 * ut):
        r, it = O.wall_newton(u, y, nu, start, tol=1e-14, maxit=10)
        assert r > 0 and it == 10
