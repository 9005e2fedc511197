"""Population storage forms against the FP64 oracle (the precision study).

LBM_FP32_DEV stores rho* and the FP32 deviations d_a = f*_a - w_a rho*; it
meets the same population gates as plain FP32 storage. LBM_FP16_DEV and
LBM_BF16_DEV keep d_a in 16 bits; for them the error against the oracle is
measured for every observable and held to the stated bounds below (about
twice the values measured on a GB300).
"""
import numpy as np
import pytest

import oracle
from paper_0708_4182_gb300 import workloads as wl
from tests.test_gpu_parity import assert_pops, check_obs, pop_err, run_both

pytestmark = pytest.mark.gpu

# stated bounds for the 16-bit forms after 100 steps:
# (relative L2 of populations, relative mass error, |dQ| / sum|u_x|/nx, rel. max|u|)
BOUNDS16 = {
    "fp16": (1e-4, 5e-8, 1e-3, 1e-3),
    "bf16": (6e-4, 5e-8, 1e-3, 5e-3),
}


@pytest.fixture(scope="module")
def lbm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0708_4182_gb300 import lbm as L
    L.load()
    return L


CASES = [
    ("droplet f=0", lambda: wl.droplet_128x64(0.0)),
    ("droplet f=0.25", lambda: wl.droplet_128x64(0.25)),
    ("rough channel", lambda: wl.rough_channel(nx=304, ny=48, amp=6, level=12, seed=5, body_fx=1e-5)),
]


@pytest.mark.parametrize("name,make", CASES)
def test_fp32_deviation_storage_meets_population_gates(lbm, name, make):
    w = make()
    p, f_ref, lat = run_both(lbm, w.mask, w.rho, w.params, 100, storage=lbm.LBM_FP32_DEV)
    assert_pops(lat.populations(), f_ref, w.mask)
    check_obs(lat, p, w.mask, f_ref)


def test_fp32_deviation_storage_tau_not_one(lbm):
    w = wl.droplet_128x64(0.15)
    params = dict(w.params, tau=0.95)
    p, f_ref, lat = run_both(lbm, w.mask, w.rho, params, 100, storage=lbm.LBM_FP32_DEV)
    assert_pops(lat.populations(), f_ref, w.mask)


@pytest.mark.parametrize("form", ["fp16", "bf16"])
@pytest.mark.parametrize("name,make", CASES)
def test_16bit_storage_errors_within_stated_bounds(lbm, form, name, make):
    w = make()
    storage = lbm.LBM_FP16_DEV if form == "fp16" else lbm.LBM_BF16_DEV
    p, f_ref, lat = run_both(lbm, w.mask, w.rho, w.params, 100, storage=storage)
    _, _, l2 = pop_err(lat.populations(), f_ref, w.mask)
    o = lat.observables()
    r = oracle.observables(p, w.mask, f_ref)
    _, ux, _ = oracle.fields(p, w.mask, f_ref)
    q_scale = np.abs(ux[w.mask == 0]).sum() / p.nx
    errs = (l2, abs(o["mass"] / r["mass"] - 1), abs(o["flux_Q"] - r["flux_Q"]) / q_scale,
            abs(o["max_u"] / r["max_u"] - 1))
    print(f"{form} {name}: L2 {errs[0]:.2e} mass {errs[1]:.2e} Q {errs[2]:.2e} max_u {errs[3]:.2e}")
    for e, b in zip(errs, BOUNDS16[form]):
        assert e <= b, (form, name, errs)


@pytest.mark.parametrize("form", ["fp16", "bf16"])
def test_16bit_storage_tau_not_one(lbm, form):
    """tau != 1: the relaxation reads g_a = f_a - w_a rho, which the FP16 form
    keeps in its raw (2^12-scaled) units. Errors against the oracle stay
    within twice the tau = 1 bounds."""
    w = wl.droplet_128x64(0.15)
    params = dict(w.params, tau=0.95)
    storage = lbm.LBM_FP16_DEV if form == "fp16" else lbm.LBM_BF16_DEV
    p, f_ref, lat = run_both(lbm, w.mask, w.rho, params, 100, storage=storage)
    _, _, l2 = pop_err(lat.populations(), f_ref, w.mask)
    o = lat.observables()
    r = oracle.observables(p, w.mask, f_ref)
    _, ux, _ = oracle.fields(p, w.mask, f_ref)
    q_scale = np.abs(ux[w.mask == 0]).sum() / p.nx
    errs = (l2, abs(o["mass"] / r["mass"] - 1), abs(o["flux_Q"] - r["flux_Q"]) / q_scale,
            abs(o["max_u"] / r["max_u"] - 1))
    print(f"{form} tau=0.95: L2 {errs[0]:.2e} mass {errs[1]:.2e} Q {errs[2]:.2e} max_u {errs[3]:.2e}")
    for e, b in zip(errs, BOUNDS16[form]):
        assert e <= 2 * b, (form, errs)


@pytest.mark.parametrize("form", ["fp32dev", "fp16", "bf16"])
def test_deviation_storage_fields_and_profile(lbm, form):
    """Density, velocity and the x-averaged u_x(y) read back from the
    deviation forms on a two-strip rough channel (the 16-bit forms' strips
    overlap): against the oracle's fields within the forms' rounding, zero
    on solid nodes, and the profile summing to the fused flux."""
    storage = {"fp32dev": lbm.LBM_FP32_DEV, "fp16": lbm.LBM_FP16_DEV, "bf16": lbm.LBM_BF16_DEV}[form]
    tol = {"fp32dev": 1e-5, "fp16": 1e-3, "bf16": 1e-2}[form]
    w = wl.rough_channel(nx=304, ny=48, amp=6, level=12, seed=5, body_fx=1e-5)
    p, f_ref, lat = run_both(lbm, w.mask, w.rho, w.params, 100, storage=storage)
    rho_g, ux_g, uy_g = lat.fields()
    rho_r, ux_r, uy_r = oracle.fields(p, w.mask, f_ref)
    solid = w.mask == 1
    assert np.all(rho_g[solid] == 0) and np.all(ux_g[solid] == 0) and np.all(uy_g[solid] == 0)
    assert np.abs(rho_g - rho_r).max() <= tol * rho_r.max()
    umax = np.abs(np.r_[ux_r.ravel(), uy_r.ravel()]).max()
    assert np.abs(ux_g - ux_r).max() <= 10 * tol * umax
    assert np.abs(uy_g - uy_r).max() <= 10 * tol * umax
    prof = lat.ux_profile()
    assert prof.sum() == pytest.approx(lat.observables()["flux_Q"], rel=1e-9, abs=1e-12)


@pytest.mark.parametrize("storage", [1, 2, 3])
def test_deviation_storage_round_trip_and_tiling(lbm, storage):
    w = wl.rough_channel(nx=304, ny=48, amp=6, level=15, seed=9, body_fx=1e-5)
    p = oracle.Params(w.nx, w.ny, **w.params)
    f0 = oracle.step(p, w.mask, oracle.equilibrium(p, w.mask, w.rho, 0, 0), 20)
    outs = []
    for tr in (4, 16, 0):
        lat = lbm.Lattice(w.nx, w.ny, storage=storage, tile_rows=tr, **w.params)
        lat.set_geometry(w.mask)
        lat.set_populations(f0)
        if tr == 4:
            back = lat.populations()
            tol = 1e-6 if storage == 1 else (2e-3 if storage == 2 else 2e-2)
            _, _, l2 = pop_err(back, f0, w.mask)
            assert l2 <= tol
        lat.step(25)
        outs.append(lat.populations())
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])


@pytest.mark.parametrize("storage", [1, 2, 3])
def test_deviation_storage_conserves_mass(lbm, storage):
    w = wl.rough_channel(nx=304, ny=48, amp=6, level=12, seed=5, body_fx=1e-5)
    lat = lbm.Lattice(w.nx, w.ny, storage=storage, **w.params)
    lat.set_geometry(w.mask)
    lat.set_rho_u(w.rho)
    m0 = lat.observables()["mass"]
    lat.step(1000)
    o = lat.observables()
    assert o["nonfinite"] == 0
    assert abs(o["mass"] / m0 - 1) <= 1e-5


RAGGED16 = [
    # nx, ny, walls, tile_rows: widths a multiple of 8 (the 16-bit forms' rule);
    # overlapping strips of 254 columns with ragged ends, an 8-column domain
    # (the staged window wraps 33 times: 34 pieces, so lanes move a second
    # piece), a single row, a single CTA
    (8, 16, True, 0),
    (16, 9, True, 4),
    (24, 30, True, 8),
    (248, 13, True, 0),
    (256, 20, True, 4),
    (512, 17, True, 0),
    (600, 1, False, 0),
]


@pytest.mark.parametrize("form", ["fp16", "bf16"])
@pytest.mark.parametrize("nx,ny,walls,tile_rows", RAGGED16)
def test_16bit_storage_ragged_and_tiny_domains(lbm, form, nx, ny, walls, tile_rows):
    """The 16-bit forms' staging (window pieces at the periodic seam, strips
    overlapping by two columns) against the oracle on ragged and tiny domains.
    A misplaced column gives errors of order 0.1 to 1. The bounds sit well
    below that and above the rounding of these blob fields after 40 steps:
    the single-row domain, the largest, measured 8.4e-4 (FP16) and 5.2e-3
    (BF16) relative L2 on a GB300, the others less."""
    from tests.test_gpu_parity import _blob_field
    mask = np.zeros((ny, nx), np.uint8)
    if walls and ny >= 3:
        mask[0] = mask[-1] = 1
        if nx >= 8 and ny >= 8:
            mask[ny // 2:ny // 2 + 2, nx // 3:nx // 3 + 3] = 1  # an interior block
    rho = _blob_field(nx, ny, mask, nx * 1000 + ny)
    params = dict(wl.PAPER, tau=1.0, f_elec=0.2, body_fx=1e-5, body_fy=-2e-6)
    storage = lbm.LBM_FP16_DEV if form == "fp16" else lbm.LBM_BF16_DEV
    p, f_ref, lat = run_both(lbm, mask, rho, params, 40, storage=storage, tile_rows=tile_rows)
    _, _, l2 = pop_err(lat.populations(), f_ref, mask)
    o = lat.observables()
    r = oracle.observables(p, mask, f_ref)
    assert o["nonfinite"] == 0
    assert l2 <= {"fp16": 2e-3, "bf16": 1e-2}[form], l2
    assert abs(o["mass"] / r["mass"] - 1) <= 1e-6


def test_16bit_storage_rejects_ragged_width(lbm):
    assert lbm.lbm_workspace_bytes(lbm.make_params(300, 48, storage=lbm.LBM_FP16_DEV)) == 0
    assert lbm.lbm_workspace_bytes(lbm.make_params(304, 48, storage=lbm.LBM_FP16_DEV)) > 0


@pytest.mark.parametrize("storage", [1, 2, 3])
def test_deviation_forms_fused_observables_and_graph_stepping(lbm, storage):
    """The deviation forms' step with fused observables gives the record of a
    separate observables pass on the same state, and one call of 75 steps
    (32-step CUDA graphs between the fused-observables steps) equals 75 calls
    of one step bitwise, with the same latest record."""
    w = wl.rough_channel(nx=304, ny=48, amp=6, level=12, seed=5, body_fx=1e-5)
    lat = lbm.Lattice(w.nx, w.ny, storage=storage, obs_every=10, **w.params)
    lat.set_geometry(w.mask)
    lat.set_rho_u(w.rho)
    lat.step(30)
    sep = lat.observables()
    lat.step(1)
    fused = lat.obs_latest()
    assert fused["step"] == sep["step"] == 30
    for k in ("mass", "flux_Q", "mom_x", "mom_y", "max_u", "min_rho"):
        assert fused[k] == pytest.approx(sep[k], rel=1e-12, abs=1e-15), k
    runs = []
    for chunks in ([75], [1] * 75):
        lat = lbm.Lattice(w.nx, w.ny, storage=storage, obs_every=10, **w.params)
        lat.set_geometry(w.mask)
        lat.set_rho_u(w.rho)
        for n in chunks:
            lat.step(n)
        runs.append((lat.populations(), lat.obs_latest()))
    assert np.array_equal(runs[0][0], runs[1][0])
    assert runs[0][1] == runs[1][1] and runs[0][1]["step"] == 70
