"""Pins of the oracle's force terms on configurations with closed forms.

Each case is derived by hand from the paper's definitions: the fluid-fluid
force (Eq. 5 with the Green function of Eq. 4), the fluid-wall force (Eq. 6),
the electric force f n on the conductive single layer next to the wall
(Eq. 9 and the critical-density paragraph), and the body force of the channel
runs. Axis and diagonal link weights are pinned separately by a profile that
varies along x and one that varies along x + y.
"""
import numpy as np
import pytest

import oracle

G = -0.52
W = -0.14


def state(p, mask, rho):
    return oracle.equilibrium(p, mask, rho, 0.0, 0.0)


def psi_of(rho):
    return 1.0 - np.exp(-rho)


@pytest.mark.parametrize("green,axis,diag", [(oracle.GREEN_MC, 1.0, 0.5),
                                             (oracle.GREEN_PRINTED, 2.0, 1.0)])
def test_sc_force_axis_profile(green, axis, diag):
    """rho = rho(x): F_x = -psi(x) (Ga + 2 Gd)(psi(x+1) - psi(x-1)), F_y = 0."""
    nx, ny = 16, 5
    x = np.arange(nx)
    rho1 = 1.0 + 0.6 * np.sin(2 * np.pi * x / nx) + 0.2 * np.cos(6 * np.pi * x / nx)
    rho = np.broadcast_to(rho1, (ny, nx)).copy()
    p = oracle.Params(nx, ny, G=G, G_wall=W, green=green)
    mask = np.zeros((ny, nx), np.uint8)
    _, _, _, t = oracle.forces(p, mask, state(p, mask, rho))
    ps = psi_of(rho1)
    expect = -ps * (axis * G + 2 * diag * G) * (np.roll(ps, -1) - np.roll(ps, 1))
    np.testing.assert_allclose(t[0], np.broadcast_to(expect, (ny, nx)), rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(t[1], 0.0, atol=1e-15)


@pytest.mark.parametrize("green,axis,diag", [(oracle.GREEN_MC, 1.0, 0.5),
                                             (oracle.GREEN_PRINTED, 2.0, 1.0)])
def test_sc_force_diagonal_profile(green, axis, diag):
    """rho = rho(s), s = x + y (mod n): F_x = F_y =
    -psi(s) [Ga (psi(s+1) - psi(s-1)) + Gd (psi(s+2) - psi(s-2))]."""
    n = 12
    s1 = np.arange(n)
    rho_s = 1.0 + 0.7 * np.sin(2 * np.pi * s1 / n)
    y, x = np.mgrid[0:n, 0:n]
    rho = rho_s[(x + y) % n]
    p = oracle.Params(n, n, G=G, green=green)
    mask = np.zeros((n, n), np.uint8)
    _, _, _, t = oracle.forces(p, mask, state(p, mask, rho))
    ps = psi_of(rho_s)
    fs = -ps * (axis * G * (np.roll(ps, -1) - np.roll(ps, 1))
                + diag * G * (np.roll(ps, -2) - np.roll(ps, 2)))
    np.testing.assert_allclose(t[0], fs[(x + y) % n], rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(t[1], fs[(x + y) % n], rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("green,axis,diag", [(oracle.GREEN_MC, 1.0, 0.5),
                                             (oracle.GREEN_PRINTED, 2.0, 1.0)])
def test_flat_wall_forces(green, axis, diag):
    """Uniform fluid between flat walls (rows 0 and ny-1 solid). On the first
    fluid row the wall force is -psi * (-(Wa + 2 Wd)) along y and the missing
    fluid neighbours leave F_sigma,y = -psi^2 (Ga + 2 Gd); mirrored on the top
    row; zero in the bulk."""
    nx, ny, r = 8, 7, 1.7
    mask = np.zeros((ny, nx), np.uint8)
    mask[0] = mask[-1] = 1
    rho = np.where(mask == 1, 0.0, r)
    p = oracle.Params(nx, ny, G=G, G_wall=W, green=green)
    _, _, _, t = oracle.forces(p, mask, state(p, mask, rho))
    ps = psi_of(r)
    k_g = axis * G + 2 * diag * G
    k_w = axis * W + 2 * diag * W
    exp_sy = np.zeros(ny)
    exp_wy = np.zeros(ny)
    exp_sy[1], exp_sy[-2] = -ps * ps * k_g, ps * ps * k_g
    exp_wy[1], exp_wy[-2] = ps * k_w, -ps * k_w
    np.testing.assert_allclose(t[1], np.broadcast_to(exp_sy[:, None], (ny, nx)), rtol=1e-14, atol=1e-15)
    np.testing.assert_allclose(t[3], np.broadcast_to(exp_wy[:, None], (ny, nx)), rtol=1e-14, atol=1e-15)
    np.testing.assert_allclose(t[0], 0.0, atol=1e-15)
    np.testing.assert_allclose(t[2], 0.0, atol=1e-15)
    # MC weights: the first-row wall force is 2 w psi, towards the wall for w < 0
    if green == oracle.GREEN_MC:
        assert t[3][1, 0] == pytest.approx(2 * W * ps, rel=1e-14)
        assert t[3][1, 0] < 0


def ewod_geometry():
    """12x8 channel (rows 0, 7 solid) with a 3-wide, 2-high step at x = 4..6."""
    nx, ny = 12, 8
    mask = np.zeros((ny, nx), np.uint8)
    mask[0] = mask[-1] = 1
    mask[1:3, 4:7] = 1
    return nx, ny, mask


def test_electric_force_layer():
    """f n acts only on conductive (rho >= rho_c) fluid nodes with a solid
    axis neighbour, one f per solid axis face, pointing into that face."""
    nx, ny, mask = ewod_geometry()
    rho = np.full((ny, nx), 1.5)
    rho[1, 1] = 0.5          # insulative vapor on the bottom layer
    rho[6, 9] = 0.5          # insulative vapor on the top layer
    rho[mask == 1] = 0.0
    fe = 0.2
    p = oracle.Params(nx, ny, G=G, G_wall=W, f_elec=fe)
    _, _, _, t = oracle.forces(p, mask, state(p, mask, rho))
    ex = np.zeros((ny, nx))
    ey = np.zeros((ny, nx))
    for x in range(nx):
        if mask[1, x] == 0:
            ey[1, x] = -fe        # bottom layer, wall below
        ey[6, x] = fe             # top layer, wall above
    ey[1, 1] = 0.0                # vapor: no force
    ey[6, 9] = 0.0
    ex[1, 3], ex[2, 3] = fe, fe   # left face of the step (solid at x = 4)
    ex[1, 7], ex[2, 7] = -fe, -fe  # right face of the step (solid at x = 6)
    ey[3, 4:7] = -fe              # top of the step (solid below)
    # (3,3) and (3,7) touch the step only diagonally: no force
    np.testing.assert_allclose(t[4], ex, atol=1e-15)
    np.testing.assert_allclose(t[5], ey, atol=1e-15)
    assert t[4][1, 3] == fe and t[5][1, 3] == -fe  # concave corner: both faces


def test_electric_force_unit_normal_reading():
    """The other reading of f n (n a unit vector): where two perpendicular
    solid faces meet, the force has length f along the diagonal instead of
    f per face; everywhere else it equals the per-face reading."""
    nx, ny, mask = ewod_geometry()
    rho = np.full((ny, nx), 1.5)
    rho[mask == 1] = 0.0
    fe = 0.2
    pf = oracle.Params(nx, ny, G=G, G_wall=W, f_elec=fe)
    pu = oracle.Params(nx, ny, G=G, G_wall=W, f_elec=fe, normal=oracle.NORMAL_UNIT)
    _, _, _, tf = oracle.forces(pf, mask, state(pf, mask, rho))
    _, _, _, tu = oracle.forces(pu, mask, state(pu, mask, rho))
    corner = (tf[4] != 0) & (tf[5] != 0)
    assert corner.sum() == 2 and corner[1, 3] and corner[1, 7]  # the step's two concave corners
    s = np.sqrt(0.5)
    assert tu[4][1, 3] == pytest.approx(fe * s, rel=1e-15) and tu[5][1, 3] == pytest.approx(-fe * s, rel=1e-15)
    assert tu[4][1, 7] == pytest.approx(-fe * s, rel=1e-15) and tu[5][1, 7] == pytest.approx(-fe * s, rel=1e-15)
    np.testing.assert_array_equal(tu[4][~corner], tf[4][~corner])
    np.testing.assert_array_equal(tu[5][~corner], tf[5][~corner])
    np.testing.assert_allclose(np.hypot(tu[4], tu[5])[tf[4] ** 2 + tf[5] ** 2 > 0], fe, rtol=1e-15)
    # the other terms do not depend on the reading
    for k in (0, 1, 2, 3, 6, 7):
        np.testing.assert_array_equal(tu[k], tf[k])


def test_unit_normal_reading_changes_nothing_on_flat_walls():
    """A droplet on a smooth wall has no node where two solid faces meet, so
    both readings give the same state step for step (the contact-angle law
    of Eq. 9 cannot tell them apart there)."""
    from paper_0708_4182_gb300 import workloads as wl
    w = wl.droplet_128x64(0.25)
    p0 = oracle.Params(w.nx, w.ny, **w.params)
    p1 = oracle.Params(w.nx, w.ny, normal=oracle.NORMAL_UNIT, **w.params)
    f0 = oracle.equilibrium(p0, w.mask, w.rho, 0, 0)
    np.testing.assert_array_equal(oracle.step(p0, w.mask, f0, 200), oracle.step(p1, w.mask, f0, 200))


def test_electric_force_threshold_is_inclusive():
    """rho == rho_c counts as conductive; the next double above does not."""
    nx, ny, mask = ewod_geometry()
    rho = np.where(mask == 1, 0.0, 1.3)
    p = oracle.Params(nx, ny, f_elec=0.1)
    f = state(p, mask, rho)
    r, _, _, _ = oracle.forces(p, mask, f)
    rc = float(r[1, 9])
    p.rho_c = rc
    _, _, _, t = oracle.forces(p, mask, f)
    assert t[5][1, 9] == -0.1
    p.rho_c = float(np.nextafter(rc, np.inf))
    _, _, _, t = oracle.forces(p, mask, f)
    assert t[5][1, 9] == 0.0


def test_body_force_is_rho_times_acceleration():
    nx, ny, mask = ewod_geometry()
    rng = np.random.default_rng(3)
    rho = np.where(mask == 1, 0.0, rng.uniform(0.1, 2.5, (ny, nx)))
    p = oracle.Params(nx, ny, body_fx=3e-5, body_fy=-1e-5)
    r, _, _, t = oracle.forces(p, mask, state(p, mask, rho))
    np.testing.assert_allclose(t[6], r * 3e-5, rtol=1e-15)
    np.testing.assert_allclose(t[7], r * -1e-5, rtol=1e-15)


def test_sc_force_pairwise_antisymmetric():
    """Eq. 5 is a sum of equal and opposite pair forces, so it sums to zero
    over the lattice, walls or not (psi = 0 on solids)."""
    from paper_0708_4182_gb300 import workloads as wl
    mask = wl.channel_mask(40, 24, amp=4, seed=7)
    rng = np.random.default_rng(5)
    rho = np.where(mask == 1, 0.0, rng.uniform(0.05, 3.0, mask.shape))
    p = oracle.Params(40, 24, G=G, G_wall=W)
    _, _, _, t = oracle.forces(p, mask, state(p, mask, rho))
    scale = np.abs(t[0]).sum() + np.abs(t[1]).sum()
    assert abs(t[0].sum()) <= 1e-13 * scale
    assert abs(t[1].sum()) <= 1e-13 * scale
    assert np.all(t[:, mask == 1] == 0)  # nothing acts on solid nodes
