"""Steady-state and long-run observables: CUDA library vs the FP64 oracle.

* Steady flux (Eq. 11): a periodic channel 128 x 40 with smooth walls,
  filled with electrolyte up to one row from each wall, driven by a body
  force of 1e-6, at electric-force levels 0, 10 and 15. Each side runs until
  |Q(t) - Q(t-1000)| / |Q(t)| < 1e-7, the rough-channel convergence criterion.
  With populations stored as deviations from the weighted rest equilibrium
  (LBM_FP32_DEV) the steady Q agree within 1e-4 relative, and Q/Q0 falls as
  f grows (the paper's flux figure). Plain FP32 storage stalls: near the
  steady state a step changes a population by less than half an ulp, the
  stored value stops moving, and Q freezes about 0.5% short; that error is
  stated and bounded here too.
* Rough-wall steady flux: a periodic 192 x 40 channel with rectangular
  roughness of height up to 4 on both walls (seed 4), liquid up to the
  crests and vapor in the grooves, body force 1e-5, electric-force levels 0
  and 6. Both sides start from the same state and run to the same criterion;
  with LBM_FP32_DEV the steady Q agree within 1e-4 relative. The vapor
  pockets in the grooves make a rough channel's steady state depend on the
  path to it, so this checks that the FP32 path follows the FP64 one to the
  same steady state, not only the same flux law.
* Contact angle: the 128 x 64 sessile droplet after 2000 steps at each of
  the five electric-force levels. cos(theta) and theta, measured on each side's
  density field with the same extractor, agree within 1e-4 relative, and
  cos(theta) rises with f (Eq. 9).
"""
import numpy as np
import pytest

import oracle
from paper_0708_4182_gb300 import workloads as wl
from tests._analysis import cos_contact_angle

pytestmark = pytest.mark.gpu

LEVELS = (0, 10, 15)
CRITERION = 1e-7


@pytest.fixture(scope="module")
def lbm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0708_4182_gb300 import lbm as L
    L.load()
    return L


def smooth_channel(level):
    return wl.rough_channel(nx=128, ny=40, amp=0, level=level, seed=3, body_fx=1e-6)


def oracle_steady(w, max_steps=80000):
    p = oracle.Params(w.nx, w.ny, **w.params)
    f = oracle.equilibrium(p, w.mask, w.rho, 0, 0)
    q_prev, t = None, 0
    while t < max_steps:
        f = oracle.step(p, w.mask, f, 1000)
        t += 1000
        q = oracle.observables(p, w.mask, f)["flux_Q"]
        if q_prev is not None and abs(q - q_prev) <= CRITERION * abs(q):
            return q, t
        q_prev = q
    raise AssertionError("oracle did not reach steady flux")


def gpu_steady(lbm, w, max_steps=80000, storage=0):
    """Through the library's own convergence loop (lbm_run_to_steady)."""
    lat = lbm.Lattice(w.nx, w.ny, storage=storage, **w.params)
    lat.set_geometry(w.mask)
    lat.set_rho_u(w.rho)
    obs, converged = lat.run_to_steady(CRITERION, 1000, max_steps)
    assert converged, "GPU run did not reach steady flux"
    assert obs["step"] == lat.time
    return obs["flux_Q"], lat.time


_ORACLE = {}


def oracle_steady_cached(level):
    if level not in _ORACLE:
        _ORACLE[level] = oracle_steady(smooth_channel(level))
    return _ORACLE[level]


def test_steady_flux_matches_oracle(lbm):
    q_gpu, q_ref = [], []
    for level in LEVELS:
        w = smooth_channel(level)
        qr, tr = oracle_steady_cached(level)
        qg, tg = gpu_steady(lbm, w, storage=lbm.LBM_FP32_DEV)
        assert qg == pytest.approx(qr, rel=1e-4), (level, qg, qr)
        # the last 1e-5-per-1000-step drift is partly below FP32 resolution, so
        # the GPU run may meet the criterion earlier (13k vs 20k steps at level 0)
        assert tg <= tr + 3000, (level, tg, tr)
        q_gpu.append(qg)
        q_ref.append(qr)
    # the paper's trend: the flux falls as the electric force grows
    assert np.all(np.diff(q_gpu) < 0) and np.all(np.diff(q_ref) < 0)
    np.testing.assert_allclose(np.array(q_gpu) / q_gpu[0], np.array(q_ref) / q_ref[0], rtol=1e-4)


ROUGH_LEVELS = (0, 6)


def rough_channel_small(level):
    return wl.rough_channel(nx=192, ny=40, amp=4, level=level, seed=4, body_fx=1e-5)


def test_rough_wall_steady_flux_matches_oracle(lbm):
    q_gpu, q_ref = [], []
    for level in ROUGH_LEVELS:
        w = rough_channel_small(level)
        qr, tr = oracle_steady(w, max_steps=80000)
        qg, tg = gpu_steady(lbm, w, max_steps=80000, storage=lbm.LBM_FP32_DEV)
        print(f"\nrough 192x40 level {level}: Q gpu {qg:.9g} ({tg} steps), oracle {qr:.9g} ({tr} steps), "
              f"rel {abs(qg / qr - 1):.2e}")
        assert qg == pytest.approx(qr, rel=1e-4), (level, qg, qr)
        assert abs(tg - tr) <= 3000, (level, tg, tr)
        q_gpu.append(qg)
        q_ref.append(qr)
    # the electric force wets the rough walls and slows the flow
    assert q_gpu[1] < q_gpu[0] and q_ref[1] < q_ref[0]


def test_contact_angle_after_2000_steps(lbm):
    cos_g, cos_r = [], []
    for fe in wl.DROPLET_F_LEVELS:
        w = wl.droplet_128x64(fe)
        p = oracle.Params(w.nx, w.ny, **w.params)
        f = oracle.step(p, w.mask, oracle.equilibrium(p, w.mask, w.rho, 0, 0), 2000)
        rho_r, _, _ = oracle.fields(p, w.mask, f)
        lat = lbm.Lattice(w.nx, w.ny, **w.params)
        lat.set_geometry(w.mask)
        lat.set_rho_u(w.rho)
        lat.step(2000)
        rho_g, _, _ = lat.fields()
        cg, _ = cos_contact_angle(rho_g, wl.RHO_L, wl.RHO_V, w.mask)
        cr, _ = cos_contact_angle(rho_r, wl.RHO_L, wl.RHO_V, w.mask)
        assert cg == pytest.approx(cr, rel=1e-4), (fe, cg, cr)
        assert np.arccos(cg) == pytest.approx(np.arccos(cr), rel=1e-4)
        cos_g.append(cg)
        cos_r.append(cr)
    assert np.all(np.diff(cos_g) > 0), cos_g


def test_steady_flux_plain_fp32_stalls_within_stated_bound(lbm):
    """Plain FP32 storage: the flux freezes before the steady state; the
    stated error bound is 1% (measured 0.50% at level 0, 0.56% at level 10)."""
    for level in (0, 10):
        qr, _ = oracle_steady_cached(level)
        qg, _ = gpu_steady(lbm, smooth_channel(level), storage=lbm.LBM_FP32)
        assert abs(qg / qr - 1) <= 1e-2, (level, qg, qr)
