"""Pins of the oracle's lattice and equilibrium (D2Q9 paragraph, Eq. 2, Eq. 3).

The velocity set is rebuilt here from the paper's trigonometric definition,
and the equilibrium is checked through its exact moments, which fix every
coefficient of Eq. 3 (weights 4/9, 1/9, 1/36 and the factors 3, 9/2, 3/2).
"""
import numpy as np
import pytest

import oracle


def paper_velocities():
    """e_0 = 0; e_a = (cos pi(a-1)/2, sin pi(a-1)/2), a = 1..4;
    e_a = sqrt(2) (cos pi(2a-1)/4, sin pi(2a-1)/4), a = 5..8."""
    e = [(0.0, 0.0)]
    for a in range(1, 5):
        t = np.pi * (a - 1) / 2
        e.append((np.cos(t), np.sin(t)))
    for a in range(5, 9):
        t = np.pi * (2 * a - 1) / 4
        e.append((np.sqrt(2) * np.cos(t), np.sqrt(2) * np.sin(t)))
    return np.rint(np.array(e)).astype(int)


def test_velocity_set_matches_paper():
    e = paper_velocities()
    assert np.array_equal(e[:, 0], oracle.EX)
    assert np.array_equal(e[:, 1], oracle.EY)
    # opposite directions
    for a in range(9):
        assert np.array_equal(e[oracle.OPP[a]], -e[a])


@pytest.fixture(scope="module")
def random_state():
    rng = np.random.default_rng(1234)
    ny, nx = 7, 11
    rho = rng.uniform(0.05, 3.0, (ny, nx))
    ux = rng.uniform(-0.2, 0.2, (ny, nx))
    uy = rng.uniform(-0.2, 0.2, (ny, nx))
    p = oracle.Params(nx, ny)
    f = oracle.equilibrium(p, np.zeros((ny, nx), np.uint8), rho, ux, uy)
    return rho, ux, uy, f


def test_rest_equilibrium_is_weights_times_rho(random_state):
    rho = random_state[0]
    ny, nx = rho.shape
    f = oracle.equilibrium(oracle.Params(nx, ny), np.zeros((ny, nx), np.uint8), rho, 0, 0)
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    np.testing.assert_allclose(f, w[:, None, None] * rho[None], rtol=1e-15, atol=0)


def test_equilibrium_moments(random_state):
    """Exact moments of the D2Q9 equilibrium:
    sum f = rho, sum f e = rho u, sum f e_i e_j = rho/3 d_ij + rho u_i u_j,
    sum f e_x^2 e_y = rho u_y / 3, sum f e_x e_y^2 = rho u_x / 3."""
    rho, ux, uy, f = random_state
    e = paper_velocities().astype(float)
    ex, ey = e[:, 0, None, None], e[:, 1, None, None]
    tol = dict(rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(f.sum(0), rho, **tol)
    np.testing.assert_allclose((f * ex).sum(0), rho * ux, **tol)
    np.testing.assert_allclose((f * ey).sum(0), rho * uy, **tol)
    np.testing.assert_allclose((f * ex * ex).sum(0), rho / 3 + rho * ux * ux, **tol)
    np.testing.assert_allclose((f * ey * ey).sum(0), rho / 3 + rho * uy * uy, **tol)
    np.testing.assert_allclose((f * ex * ey).sum(0), rho * ux * uy, **tol)
    np.testing.assert_allclose((f * ex * ex * ey).sum(0), rho * uy / 3, **tol)
    np.testing.assert_allclose((f * ex * ey * ey).sum(0), rho * ux / 3, **tol)


def test_equilibrium_zero_on_solid():
    p = oracle.Params(3, 3)
    mask = np.zeros((3, 3), np.uint8)
    mask[1, 1] = 1
    f = oracle.equilibrium(p, mask, 1.0, 0.1, 0.0)
    assert np.all(f[:, 1, 1] == 0)
    assert np.all(f[:, 0, 0] > 0)


def test_fields_of_equilibrium_state():
    """A resting uniform fluid has zero force, so rho and u come back exactly."""
    ny, nx = 5, 6
    p = oracle.Params(nx, ny, G=-0.52, G_wall=0.0)
    mask = np.zeros((ny, nx), np.uint8)
    f = oracle.equilibrium(p, mask, 0.85, 0.0, 0.0)
    rho, ux, uy = oracle.fields(p, mask, f)
    np.testing.assert_allclose(rho, 0.85, rtol=1e-15)
    np.testing.assert_allclose(ux, 0.0, atol=1e-16)
    np.testing.assert_allclose(uy, 0.0, atol=1e-16)


def test_equilibrium_physical_round_trip():
    """The state built for a physical velocity u reads back, through the
    separately pinned fields() (u = (j + F/2)/rho), as exactly (rho, u):
    random density with a liquid/vapor mix, rough walls, electric and body
    force all active."""
    rng = np.random.default_rng(3)
    ny, nx = 12, 16
    mask = np.zeros((ny, nx), np.uint8)
    mask[0, :] = mask[-1, :] = 1
    mask[1, 3:6] = 1
    p = oracle.Params(nx, ny, tau=1.0, G=-0.52, G_wall=-0.14, f_elec=0.2, body_fx=1e-3, body_fy=-2e-4)
    rho = np.where(rng.random((ny, nx)) < 0.5, 2.8, 0.07) * (1 + 0.05 * rng.standard_normal((ny, nx)))
    ux = 0.02 * rng.standard_normal((ny, nx))
    uy = 0.02 * rng.standard_normal((ny, nx))
    f = oracle.equilibrium_physical(p, mask, rho, ux, uy)
    r2, u2, v2 = oracle.fields(p, mask, f)
    fl = mask == 0
    np.testing.assert_allclose(r2[fl], rho[fl], rtol=1e-14)
    np.testing.assert_allclose(u2[fl], ux[fl], rtol=0, atol=1e-13)
    np.testing.assert_allclose(v2[fl], uy[fl], rtol=0, atol=1e-13)
    # and the force shift is not trivial here
    plain = oracle.equilibrium(p, mask, rho, ux, uy)
    assert np.max(np.abs(plain - f)) > 1e-3


def test_equilibrium_physical_body_force_only():
    """With only a body force, F = rho f_b and the equilibrium velocity is
    u - f_b/2 at every node (no walls)."""
    ny, nx = 4, 6
    p = oracle.Params(nx, ny, G=0.0, G_wall=0.0, body_fx=4e-3, body_fy=-1e-3)
    mask = np.zeros((ny, nx), np.uint8)
    f = oracle.equilibrium_physical(p, mask, 1.3, 0.01, 0.02)
    ref = oracle.equilibrium(p, mask, 1.3, 0.01 - 2e-3, 0.02 + 5e-4)
    np.testing.assert_allclose(f, ref, rtol=1e-15, atol=1e-17)
