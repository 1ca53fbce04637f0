"""Pins of the oracle's local cell model (no GPU).

Each test ties the FP64 oracle to something other than itself: lattice
quadrature identities, Maxwellian moments that the third-order equilibrium
must reproduce, Hermite projection identities, the defining implicit
equation of the Smagorinsky relaxation time, and the moment-level statement
of the (hybrid) regularized collision.
"""

import numpy as np
import pytest

import oracle as O
from workloads import random_populations

CS2 = 1.0 / 3.0
I3 = np.eye(3)


@pytest.mark.parametrize("q", [19, 27])
def test_lattice_quadrature(q):
    """Velocity set and weights (Fig. D3Q19 / the D3Q27 product lattice):
    zeroth, second and fourth moments are isotropic with cs^2 = 1/3, odd
    moments vanish; these conditions fix the weights uniquely."""
    c, w, opp = O.lattice(q)
    full = {(a, b, g) for a in (-1, 0, 1) for b in (-1, 0, 1) for g in (-1, 0, 1)}
    want = {v for v in full if sum(x * x for x in v) <= (2 if q == 19 else 3)}
    assert {tuple(v) for v in c} == want
    assert np.all(c[opp] == -c)
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.allclose(np.einsum("i,ia->a", w, c), 0.0, atol=1e-16)
    assert np.allclose(np.einsum("i,ia,ib->ab", w, c, c), CS2 * I3, atol=1e-15)
    assert np.allclose(np.einsum("i,ia,ib,ig->abg", w, c, c, c), 0.0, atol=1e-16)
    M4 = np.einsum("i,ia,ib,ig,id->abgd", w, c, c, c, c)
    iso = CS2**2 * (np.einsum("ab,gd->abgd", I3, I3) + np.einsum("ag,bd->abgd", I3, I3)
                    + np.einsum("ad,bg->abgd", I3, I3))
    assert np.allclose(M4, iso, atol=1e-15)
    if q == 27:
        # sixth-order isotropy of the product lattice: sum w cx^2 cy^2 cz^2 = cs^6
        assert abs(np.sum(w * c[:, 0] ** 2 * c[:, 1] ** 2 * c[:, 2] ** 2) - CS2**3) < 1e-16
    rest = np.where((c == 0).all(1))[0][0]
    assert abs(w[rest] - (1 / 3 if q == 19 else 8 / 27)) < 1e-16


def _maxwell_third(rho, u):
    """Third moment of a Maxwellian: rho cs2 (u_a d_bg + u_b d_ag + u_g d_ab) + rho u_a u_b u_g."""
    return (rho * CS2 * (np.einsum("a,bg->abg", u, I3) + np.einsum("b,ag->abg", u, I3)
                         + np.einsum("g,ab->abg", u, I3)) + rho * np.einsum("a,b,g->abg", u, u, u))


@pytest.mark.parametrize("q", [19, 27])
def test_equilibrium_moments(q):
    """Third-order equilibrium (Sec. 2.2): mass, momentum and the full second
    moment of a Maxwellian are exact; the mixed third moments are exact on
    D3Q27, and on D3Q19 they carry the known aliasing of H_xxy with H_yzz
    (<H_xxy H_yzz> = -cs^6 on D3Q19), which pins the 1/(3! cs^6) factor."""
    c, w, _ = O.lattice(q)
    rng = np.random.default_rng(1)
    for _ in range(25):
        rho = 1.0 + 0.1 * rng.uniform(-1, 1)
        u = rng.uniform(-0.15, 0.15, 3)
        feq = O.equilibrium(q, rho, u)
        assert abs(feq.sum() - rho) < 1e-14
        assert np.allclose(c.T @ feq, rho * u, atol=1e-15)
        M2 = np.einsum("i,ia,ib->ab", feq, c, c)
        assert np.allclose(M2, rho * CS2 * I3 + rho * np.outer(u, u), atol=1e-15)
        M3 = np.einsum("i,ia,ib,ig->abg", feq, c, c, c)
        ref = _maxwell_third(rho, u)
        for a in range(3):
            for b in range(3):
                for g in range(3):
                    if a == b == g:
                        # c_a^3 = c_a on these lattices: the diagonal third moment is rho u_a
                        assert abs(M3[a, b, g] - rho * u[a]) < 1e-15
                        continue
                    if q == 27:
                        assert abs(M3[a, b, g] - ref[a, b, g]) < 1e-15
                    elif len({a, b, g}) == 3:
                        assert abs(M3[a, b, g]) < 1e-16
                    else:
                        # the pair index p (twice) and single index s: xxy -> p=x, s=y
                        idx = [a, b, g]
                        s = [k for k in idx if idx.count(k) == 1][0]
                        p = [k for k in idx if idx.count(k) == 2][0]
                        o = 3 - s - p
                        want = rho * CS2 * u[s] + rho * u[p] ** 2 * u[s] - 0.5 * rho * u[s] * u[o] ** 2
                        assert abs(M3[a, b, g] - want) < 1e-15


@pytest.mark.parametrize("q", [19, 27])
def test_regularized_projection(q):
    """f^(1) (Sec. 2.2) carries no mass or momentum and its second moment is a1^(2)."""
    c, w, _ = O.lattice(q)
    rng = np.random.default_rng(2)
    for _ in range(25):
        A = rng.normal(size=(3, 3)) * 1e-3
        a2 = A + A.T
        u = rng.uniform(-0.1, 0.1, 3)
        f1 = O.regularized_neq(q, a2, u)
        assert abs(f1.sum()) < 1e-17
        assert np.allclose(c.T @ f1, 0.0, atol=1e-17)
        assert np.allclose(np.einsum("i,ia,ib->ab", f1, c, c), a2, atol=1e-16)
        if q == 27:
            # D3Q27 resolves the mixed third-order Hermite moments exactly
            M3 = np.einsum("i,ia,ib,ig->abg", f1, c, c, c)
            a3 = (np.einsum("a,bg->abg", u, a2) + np.einsum("b,ag->abg", u, a2)
                  + np.einsum("g,ab->abg", u, a2))
            for a in range(3):
                for b in range(3):
                    for g in range(3):
                        if not a == b == g:
                            assert abs(M3[a, b, g] - a3[a, b, g]) < 1e-17


def test_smagorinsky_implicit_equation():
    """Eqs. (turbVisc) and (tauEff) with dx = dt = 1: tau = tau_mo + 3 C_S^2 |S|,
    where the strain rate follows from the non-equilibrium stress as
    S = -Pi_neq / (2 rho cs^2 tau) and |S| = sqrt(2 S:S)."""
    rng = np.random.default_rng(3)
    for _ in range(50):
        A = rng.normal(size=(3, 3)) * 10 ** rng.uniform(-6, -2)
        P = A + A.T
        rho = 1 + 0.05 * rng.uniform(-1, 1)
        tau_mo = rng.uniform(0.5001, 1.5)
        cs = rng.uniform(0.0, 0.2)
        tau = O.smagorinsky_tau(tau_mo, cs, rho, P)
        S = -P / (2 * rho * CS2 * tau)
        Smag = np.sqrt(2 * np.sum(S * S))
        assert abs(tau - (tau_mo + 3 * cs**2 * Smag)) < 1e-13 * tau
        assert tau >= tau_mo
    assert O.smagorinsky_tau(0.7, 0.0, 1.0, np.ones((3, 3))) == 0.7


@pytest.mark.parametrize("q", [19, 27])
def test_collision_moments(q):
    """Collision, Eq. (hlbm) with the hybrid f~(1): mass is conserved, the
    momentum becomes rho u^ with u^ = d u + (1 - d) u^B (Eq. convexVelocity,
    d = 1 in fluid), and the second moment is
    rho cs2 I + rho u^ u^ + (1 - 1/tau) (sigma Pi_neq - (1 - sigma) 2 rho cs2 tau S_FD)."""
    c, w, _ = O.lattice(q)
    n = 400
    f = random_populations(11, n, w, amplitude=0.08)
    rng = np.random.default_rng(4)
    d = rng.uniform(0, 1, n)
    d[:40] = 1.0
    d[40:80] = 0.0
    uB = rng.uniform(-0.2, 0.2, (n, 3))
    sigma = rng.uniform(0, 1, n)
    sigma[:20] = 1.0
    sigma[80:100] = 0.0
    A = rng.normal(size=(n, 3, 3)) * 1e-3
    Sfd = A + np.transpose(A, (0, 2, 1))
    fout, tau = O.collide_cells(q, f, d, uB, sigma, Sfd, tau_mo=0.52, c_smag=0.14)
    rho = f.sum(1)
    u = (f @ c) / rho[:, None]
    uh = d[:, None] * u + (1 - d[:, None]) * uB
    assert np.allclose(fout.sum(1), rho, rtol=0, atol=1e-15)
    assert np.allclose(fout @ c, rho[:, None] * uh, rtol=0, atol=1e-15)
    Pi = np.einsum("ni,ia,ib->nab", f, c, c)
    Pneq = Pi - rho[:, None, None] * CS2 * I3 - rho[:, None, None] * np.einsum("na,nb->nab", u, u)
    Pout = np.einsum("ni,ia,ib->nab", fout, c, c)
    r3 = rho[:, None, None]
    t3 = tau[:, None, None]
    s3 = sigma[:, None, None]
    want = (r3 * CS2 * I3 + r3 * np.einsum("na,nb->nab", uh, uh)
            + (1 - 1 / t3) * (s3 * Pneq - (1 - s3) * 2 * r3 * CS2 * t3 * Sfd))
    assert np.allclose(Pout, want, rtol=0, atol=2e-15)
    # d = 0: the cell is driven to the solid velocity exactly
    v = (fout[40:80] @ c) / fout[40:80].sum(1)[:, None]
    assert np.allclose(v, uB[40:80], rtol=0, atol=1e-15)
    # the relaxation time is the Smagorinsky root of each cell's own stress
    for k in range(0, n, 37):
        assert abs(tau[k] - O.smagorinsky_tau(0.52, 0.14, rho[k], Pneq[k])) < 1e-15


def test_collision_rest_and_bulk_equivalence():
    """A band cell with d = 1 and sigma = 1 collides exactly like a bulk cell
    (RRLBM-LES), whatever u^B and S_FD are; the rest state is a fixed point."""
    c, w, _ = O.lattice(19)
    f = random_populations(5, 64, w, amplitude=0.05)
    a, _ = O.collide_cells(19, f)
    b, _ = O.collide_cells(19, f, d=np.ones(64), uB=np.full((64, 3), 0.3), sigma=np.ones(64),
                           Sfd=np.full((64, 3, 3), 0.01))
    assert np.array_equal(a, b)
    r, _ = O.collide_cells(19, np.tile(w, (3, 1)))
    assert np.allclose(r, w, rtol=0, atol=1e-15)
