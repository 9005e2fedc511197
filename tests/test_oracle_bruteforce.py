"""Brute-force pin of one whole oracle step on tiny lattices.

An independent restatement of one time step in 50-digit arithmetic (mpmath),
node by node from the paper's definitions:
  moments (Eq. 2); psi = rho0 (1 - exp(-rho/rho0)); fluid-fluid force (Eq. 5)
  with psi = 0 on solids; fluid-wall force (Eq. 6); the electric force f per
  solid axis face on conductive (rho >= rho_c) nodes; the body force rho f_b;
  the shifted velocity of Eq. 10; BGK relaxation to Eq. 3 (Eq. 1); streaming
  with half-way bounce-back.
Unlike the oracle it pulls (f_a(x) = f*_a(x - e_a), or f*_opp(a)(x) if
x - e_a is solid), takes the velocity set from the paper's trigonometric
definition and finds opposite directions by search. The oracle's FP64 step
must agree to 1e-13 relative: a dropped term, a wrong sign, a transposed
index or a wrong weight anywhere in the step shows up far above that.
"""
import itertools

import numpy as np
import pytest

import oracle

mp = pytest.importorskip("mpmath")

mp.mp.dps = 50


def velocity_set():
    e = [(0, 0)]
    for a in range(1, 5):
        t = mp.pi * (a - 1) / 2
        e.append((int(mp.nint(mp.cos(t))), int(mp.nint(mp.sin(t)))))
    for a in range(5, 9):
        t = mp.pi * (2 * a - 1) / 4
        e.append((int(mp.nint(mp.sqrt(2) * mp.cos(t))), int(mp.nint(mp.sqrt(2) * mp.sin(t)))))
    return e


E = velocity_set()
OPP = [E.index((-ex, -ey)) for ex, ey in E]
W = [mp.mpf(4) / 9] + [mp.mpf(1) / 9] * 4 + [mp.mpf(1) / 36] * 4


def exact_step(f, solid, prm):
    """f: dict (a, x, y) -> mpf post-streaming populations; returns the same at t + 1."""
    ny, nx = solid.shape
    tau, G, Gw = prm["tau"], prm["G"], prm["G_wall"]
    rho0, rho_c, fe, bfx, bfy = prm["rho0"], prm["rho_c"], prm["f_elec"], prm["body_fx"], prm["body_fy"]
    # Martys-Chen magnitudes: G on |e| = 1 links, G/2 on |e| = sqrt 2 links; W_a likewise
    Ga = [0] + [G] * 4 + [G / 2] * 4
    Wa = [0] + [Gw] * 4 + [Gw / 2] * 4
    nodes = [(x, y) for y in range(ny) for x in range(nx)]
    fluid = {(x, y): solid[y, x] == 0 for x, y in nodes}
    rho = {n: sum(f[(a, *n)] for a in range(9)) if fluid[n] else mp.mpf(0) for n in nodes}
    psi = {n: rho0 * (1 - mp.exp(-rho[n] / rho0)) if fluid[n] else mp.mpf(0) for n in nodes}

    def nb(n, a):
        return ((n[0] + E[a][0]) % nx, (n[1] + E[a][1]) % ny)

    fstar = {}
    for n in nodes:
        if not fluid[n]:
            continue
        jx = sum(f[(a, *n)] * E[a][0] for a in range(9))
        jy = sum(f[(a, *n)] * E[a][1] for a in range(9))
        Fx = Fy = mp.mpf(0)
        for a in range(1, 9):
            m = nb(n, a)
            s = 0 if fluid[m] else 1
            Fx += -psi[n] * (Ga[a] * psi[m] + Wa[a] * s) * E[a][0]
            Fy += -psi[n] * (Ga[a] * psi[m] + Wa[a] * s) * E[a][1]
        if rho[n] >= rho_c:
            for a in range(1, 5):
                if not fluid[nb(n, a)]:
                    Fx += fe * E[a][0]
                    Fy += fe * E[a][1]
        Fx += rho[n] * bfx
        Fy += rho[n] * bfy
        ux = (jx + tau * Fx) / rho[n]
        uy = (jy + tau * Fy) / rho[n]
        for a in range(9):
            c = E[a][0] * ux + E[a][1] * uy
            feq = W[a] * rho[n] * (1 + 3 * c + mp.mpf(9) / 2 * c * c - mp.mpf(3) / 2 * (ux * ux + uy * uy))
            fstar[(a, *n)] = f[(a, *n)] - (f[(a, *n)] - feq) / tau
    out = {}
    for n in nodes:
        for a in range(9):
            if not fluid[n]:
                out[(a, *n)] = mp.mpf(0)
                continue
            src = ((n[0] - E[a][0]) % nx, (n[1] - E[a][1]) % ny)
            out[(a, *n)] = fstar[(a, *src)] if fluid[src] else fstar[(OPP[a], *n)]
    return out


CASES = {
    "4x4 solid bottom row": (4, 4, [(x, 0) for x in range(4)]),
    "5x3 two solid nodes": (5, 3, [(2, 1), (0, 0)]),
    "6x5 channel with a step": (6, 5, [(x, 0) for x in range(6)] + [(x, 4) for x in range(6)] + [(2, 1), (3, 1)]),
}


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("tau", ["1", "0.9", "1.3"])
def test_one_step_matches_exact_arithmetic(name, tau):
    nx, ny, solids = CASES[name]
    solid = np.zeros((ny, nx), np.uint8)
    for x, y in solids:
        solid[y, x] = 1
    rng = np.random.default_rng(nx * 100 + ny)
    # liquid-like and vapor-like nodes so that the rho >= rho_c test splits them
    base = np.where(rng.random((ny, nx)) < 0.5, 2.6, 0.08)
    f = (base[None] / 9) * (0.6 + 0.8 * rng.random((9, ny, nx)))
    f[:, solid == 1] = 0.0
    prm = dict(tau=float(tau), G=-0.52, G_wall=-0.14, rho0=1.0, rho_c=1.0, f_elec=0.125,
               body_fx=1e-3, body_fy=-5e-4)
    p = oracle.Params(nx, ny, **prm)
    got = oracle.step(p, solid, f, 1)
    exact_prm = {k: mp.mpf(str(v)) for k, v in prm.items()}
    fe = {(a, x, y): mp.mpf(float(f[a, y, x])) for a, x, y in itertools.product(range(9), range(nx), range(ny))}
    ref = exact_step(fe, solid, exact_prm)
    ref_arr = np.array([[[float(ref[(a, x, y)]) for x in range(nx)] for y in range(ny)] for a in range(9)])
    scale = np.abs(ref_arr).max()
    assert np.abs(got - ref_arr).max() <= 1e-13 * scale
    # the case exercises every force: the electric and wall terms are not zero
    assert (solid == 0).any() and (base[solid == 0] > 1).any()


def test_bruteforce_detects_a_planted_error():
    """A planted weight error in the oracle (the printed 2G/G Green weights
    instead of G/G/2) lands far outside the agreement bound, so the bound
    has teeth."""
    nx, ny, solids = CASES["4x4 solid bottom row"]
    solid = np.zeros((ny, nx), np.uint8)
    for x, y in solids:
        solid[y, x] = 1
    rng = np.random.default_rng(7)
    f = (np.where(rng.random((ny, nx)) < 0.5, 2.6, 0.08)[None] / 9) * (0.6 + 0.8 * rng.random((9, ny, nx)))
    f[:, solid == 1] = 0.0
    prm = dict(tau=1.0, G=-0.52, G_wall=-0.14, rho0=1.0, rho_c=1.0, f_elec=0.125, body_fx=1e-3, body_fy=0.0)
    got = oracle.step(oracle.Params(nx, ny, **prm), solid, f, 1)
    # plant: the printed-weight convention (2G axis, G diagonal) in the oracle
    bad = oracle.step(oracle.Params(nx, ny, green=oracle.GREEN_PRINTED, **prm), solid, f, 1)
    exact_prm = {k: mp.mpf(str(v)) for k, v in prm.items()}
    fe = {(a, x, y): mp.mpf(float(f[a, y, x])) for a, x, y in itertools.product(range(9), range(nx), range(ny))}
    ref = exact_step(fe, solid, exact_prm)
    ref_arr = np.array([[[float(ref[(a, x, y)]) for x in range(nx)] for y in range(ny)] for a in range(9)])
    scale = np.abs(ref_arr).max()
    assert np.abs(got - ref_arr).max() <= 1e-13 * scale
    assert np.abs(bad - ref_arr).max() > 1e-4 * scale
