"""Warm start from the trained U-Net surrogate.

The surrogate is trained on the GPU, by the hand-written kernels, on steady
states that the method itself produces (flat-wall channels of varying
height, electric-force level and fill). Its prediction initialises a batched
run through LBM_RHO_U_PHYS, and the method runs on to its usual convergence
criterion (|dQ|/|Q| < 1e-7 per 1000 steps), so the surrogate's error is
measured by the converged flux: every warm-started channel must reach the
cold start's steady flux within 1e-3, in fewer steps than the cold start.
Rough-wall channels keep their cold start (their steady flux depends on the
path, through where vapor pockets settle) and must come out exactly as the
cold run.
"""
import numpy as np
import pytest

from paper_0708_4182_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def trained():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0708_4182_gb300 import lbm as L, surrogate as S
    L.load()
    S.load_unet()
    net, info = S.fit(wl.smooth_channels(512, seed=100), epochs=25)
    return S, net, info


def test_training_converges(trained):
    S, net, info = trained
    assert info["samples"] == 512
    assert info["loss"][-1] < 0.05 * info["loss"][0], info["loss"]


def test_untrained_network_falls_back(trained):
    """An untrained network's prediction is far from steady: the probe
    finds a residual that does not fall below the fallback threshold and the
    domain restarts from its cold start, so the converged flux is still the
    cold start's."""
    S, _, _ = trained
    raw = S.UNet(batch=16, height=64, width=256, seed=3)
    raw.norm = dict(rho_mean=1.5, rho_std=1.0, u_scale=0.1)
    ws = wl.smooth_channels(4, seed=13)
    cold_steps, cold_obs, _ = S.batch_run_to_steady(ws)
    steps, obs, info = S.batch_run_to_steady(ws, raw)
    for i in range(4):
        if info["restarted"][i]:
            assert steps[i] == cold_steps[i] + 2000
            assert obs[i]["flux_Q"] == cold_obs[i]["flux_Q"]
        else:
            assert steps[i] > 0
            assert abs(obs[i]["flux_Q"] / cold_obs[i]["flux_Q"] - 1) <= 1e-3


def test_warm_start_saves_steps_at_unchanged_flux(trained):
    S, net, _ = trained
    ws = wl.smooth_channels(16, seed=7)
    cold_steps, cold_obs, info0 = S.batch_run_to_steady(ws)
    assert not any(info0["warm"]) and min(cold_steps) > 0
    steps, obs, info = S.batch_run_to_steady(ws, net)
    assert all(info["warm"]) and not any(info["restarted"]), info["probe_residuals"]
    assert min(steps) > 0
    q_cold = np.array([o["flux_Q"] for o in cold_obs])
    q_warm = np.array([o["flux_Q"] for o in obs])
    assert np.all(np.abs(q_warm / q_cold - 1) <= 1e-3), np.abs(q_warm / q_cold - 1)
    assert sum(steps) <= 0.8 * sum(cold_steps), (sum(steps), sum(cold_steps))


def test_rough_domains_keep_the_cold_start(trained):
    S, net, _ = trained
    flat = wl.smooth_channels(2, seed=21)
    rough = [wl.rough_channel(nx=256, ny=64, amp=a, level=lv, seed=sd, body_fx=1e-5)
             for a, lv, sd in ((6, 3, 5), (4, 12, 8))]
    ws = [flat[0], rough[0], flat[1], rough[1]]
    steps, obs, info = S.batch_run_to_steady(ws, net)
    assert info["warm"] == [True, False, True, False]
    cold_steps, cold_obs, _ = S.batch_run_to_steady(ws)
    for i in (1, 3):
        if cold_steps[i] > 0:
            assert steps[i] == cold_steps[i]
            assert obs[i]["flux_Q"] == cold_obs[i]["flux_Q"]


def test_rough_walls_steady_flux_depends_on_the_path():
    """Why rough walls keep their cold start, and why warm starts go through
    LBM_RHO_U_PHYS: four rough channels run to steady flux and restart from
    their own converged (rho, u). Restarted as f_eq(rho, u) (a momentum kick
    of F/2 per node at every interface) at least one settles on another
    steady flux; restarted with the force correction every one returns to
    its flux within 1e-3 after a few thousand steps."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0708_4182_gb300 import lbm as L
    L.load()
    ws = [wl.warm_start_channels(32, seed=7)[i] for i in (11, 17, 18, 22)]
    specs = [dict(nx=w.nx, ny=w.ny, storage=L.LBM_FP32_DEV, **w.params) for w in ws]

    def run(setter):
        b = L.Batch(specs)
        for i, (w, d) in enumerate(zip(ws, b.domains)):
            d.set_geometry(w.mask)
            setter(i, w, d)
        steps, obs, _ = b.run_to_steady(1e-7, 1000, 80000)
        fields = [d.fields_device() for d in b.domains]
        b.close()
        return np.array(steps), np.array([o["flux_Q"] for o in obs]), fields

    cold_steps, q_cold, f_cold = run(lambda i, w, d: d.set_rho_u(w.rho))
    assert np.all(cold_steps > 0)
    _, q_kick, _ = run(lambda i, w, d: d.set_rho_u_field(f_cold[i]))
    phys_steps, q_phys, _ = run(lambda i, w, d: d.set_rho_u_field(f_cold[i], physical=True))
    rel_kick = np.abs(q_kick / q_cold - 1)
    rel_phys = np.abs(q_phys / q_cold - 1)
    assert np.all(rel_phys <= 1e-3), rel_phys
    assert np.all((phys_steps > 0) & (phys_steps <= 10000)), phys_steps
    assert rel_kick.max() > 3e-3, rel_kick
