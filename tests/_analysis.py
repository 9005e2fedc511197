"""Contact-angle measurement used by the tests on any density field.

The paper reads the contact angle off its droplet figures without saying how
(no method is given with its droplet results). The tests measure it the same
way on every field they compare, whether the field came from the oracle or
from the CUDA library:

* interface points are where the density crosses the mid level
  (rho_l + rho_v)/2, linearly interpolated along rows and columns;
* points closer than ``y_min`` to the bottom wall row are dropped (the wall
  force distorts the profile there);
* a Kasa least-squares circle x^2 + y^2 = 2 a x + 2 b y + c is fitted;
* with the wall plane at y = 0.5 (half-way bounce-back above a solid row 0),
  cos(theta) = -(b - 0.5)/R, theta measured through the liquid.
"""
import numpy as np


def interface_points(rho, level, mask=None, y_min=3.5):
    ny, nx = rho.shape
    fluid = np.ones_like(rho, dtype=bool) if mask is None else (mask == 0)
    pts = []
    a, b = rho[:, :-1], rho[:, 1:]
    ok = fluid[:, :-1] & fluid[:, 1:] & ((a - level) * (b - level) < 0)
    ys, xs = np.nonzero(ok)
    t = (level - a[ys, xs]) / (b[ys, xs] - a[ys, xs])
    pts.append(np.stack([xs + t, ys.astype(float)], 1))
    a, b = rho[:-1, :], rho[1:, :]
    ok = fluid[:-1, :] & fluid[1:, :] & ((a - level) * (b - level) < 0)
    ys, xs = np.nonzero(ok)
    t = (level - a[ys, xs]) / (b[ys, xs] - a[ys, xs])
    pts.append(np.stack([xs.astype(float), ys + t], 1))
    p = np.concatenate(pts)
    return p[p[:, 1] >= y_min]


def fit_circle(pts):
    x, y = pts[:, 0], pts[:, 1]
    A = np.c_[2 * x, 2 * y, np.ones_like(x)]
    sol = np.linalg.lstsq(A, x * x + y * y, rcond=None)[0]
    xc, yc = sol[0], sol[1]
    return xc, yc, float(np.sqrt(sol[2] + xc * xc + yc * yc))


def cos_contact_angle(rho, rho_l, rho_v, mask=None, wall_y=0.5, y_min=3.5):
    """cos(theta) of a sessile droplet on the bottom wall, and the fit."""
    pts = interface_points(rho, 0.5 * (rho_l + rho_v), mask, y_min)
    xc, yc, R = fit_circle(pts)
    return -(yc - wall_y) / R, (xc, yc, R)
