"""Pins of the oracle's observables (Eq. 11 and the bookkeeping values).

A hand-built state fixes every output exactly. With G = G_wall = f = 0 the
only force is the body force, F = rho b, so a node whose populations are
Eq. 3's equilibrium at (rho_i, u_i) has density rho_i and physical velocity
(sum f e + F/2)/rho = u_i + b/2 (the velocity of Eq. 11, reading R7), by the
exact moments of the equilibrium. The expected values below come from rho_i
and u_i alone:

* max |u| is taken over the physical velocity of fluid nodes: the node
  with the largest |u_i| is not the one with the largest |u_i + b/2|, and the
  shifted velocity u_i + tau b of Eq. 10 has its maximum at a third value;
* min rho is taken over fluid nodes: every solid node holds a smaller density
  (and a larger velocity) than any fluid node, which must not count;
* a fluid node enclosed by solids holds NaN populations: it is counted as
  non-finite and enters none of the sums, the maximum or the minimum.
"""
import numpy as np
import pytest

import oracle

EX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
EY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


def feq(rho, ux, uy):
    """Eq. 3 written out per direction (the state builder of this test)."""
    c = EX[:, None, None] * ux + EY[:, None, None] * uy
    return W[:, None, None] * rho * (1 + 3 * c + 4.5 * c * c - 1.5 * (ux * ux + uy * uy))


def _state(nan_cell=True):
    nx, ny = 12, 9
    rng = np.random.default_rng(41)
    rho = rng.uniform(0.6, 1.4, (ny, nx))
    ux = rng.uniform(-0.03, 0.03, (ny, nx))
    uy = rng.uniform(-0.03, 0.03, (ny, nx))
    mask = np.zeros((ny, nx), np.uint8)
    mask[0, :] = 1                        # a wall row
    mask[3:6, 8:11] = 1                   # a solid ring around (x=9, y=4)
    mask[4, 9] = 0
    # node B has the largest physical speed, node A the largest raw speed
    ux[2, 3], uy[2, 3] = -0.06, 0.0       # A
    ux[6, 5], uy[6, 5] = 0.045, 0.0       # B
    rho[7, 1] = 0.37                      # the smallest fluid density
    # solids carry a smaller density and a larger velocity than any fluid node
    rho = np.where(mask == 1, 0.01, rho)
    ux = np.where(mask == 1, 0.9, ux)
    f = feq(rho, ux, uy)
    if nan_cell:
        f[:, 4, 9] = np.nan
    return mask, rho, ux, uy, f


def test_observables_of_a_hand_built_state():
    mask, rho, ux, uy, f = _state()
    bx, by = 0.02, -0.01
    ny, nx = mask.shape
    p = oracle.Params(nx, ny, tau=0.9, G=0.0, G_wall=0.0, f_elec=0.0, body_fx=bx, body_fy=by)
    o = oracle.observables(p, mask, f)
    fl = mask == 0
    fl[4, 9] = False                      # the NaN cell
    vx, vy = ux[fl] + bx / 2, uy[fl] + by / 2
    speed = np.hypot(vx, vy)
    assert o["nonfinite"] == 1
    assert o["max_u"] == pytest.approx(speed.max(), rel=1e-12)
    assert o["max_u"] == pytest.approx(np.hypot(0.045 + bx / 2, by / 2), rel=1e-12)
    # neither the raw j/rho nor the shifted u' = u + tau F/rho gives it
    assert abs(o["max_u"] - np.hypot(ux[fl], uy[fl]).max()) > 1e-3
    assert abs(o["max_u"] - np.hypot(ux[fl] + 0.9 * bx, uy[fl] + 0.9 * by).max()) > 1e-3
    assert o["min_rho"] == pytest.approx(0.37, rel=1e-12)
    assert o["mass"] == pytest.approx(rho[fl].sum(), rel=1e-12)
    assert o["flux_Q"] == pytest.approx(vx.sum() / nx, rel=1e-12)
    assert o["mom_x"] == pytest.approx((rho[fl] * vx).sum(), rel=1e-12)
    assert o["mom_y"] == pytest.approx((rho[fl] * vy).sum(), rel=1e-12)


def test_fields_match_the_hand_built_velocity():
    """The per-node fields behind the observables: rho_i and u_i + b/2 on
    fluid nodes, zero velocity on solids."""
    mask, rho, ux, uy, f = _state(nan_cell=False)
    bx, by = 0.02, -0.01
    ny, nx = mask.shape
    p = oracle.Params(nx, ny, tau=1.0, G=0.0, G_wall=0.0, f_elec=0.0, body_fx=bx, body_fy=by)
    r, vx, vy = oracle.fields(p, mask, f)
    fl = mask == 0
    np.testing.assert_allclose(r[fl], rho[fl], rtol=1e-13)
    np.testing.assert_allclose(vx[fl], ux[fl] + bx / 2, rtol=0, atol=1e-14)
    np.testing.assert_allclose(vy[fl], uy[fl] + by / 2, rtol=0, atol=1e-14)
    assert np.all(vx[~fl] == 0) and np.all(vy[~fl] == 0)
    o = oracle.observables(p, mask, f)
    assert o["nonfinite"] == 0
    assert o["min_rho"] == pytest.approx(rho[fl].min(), rel=1e-12)
