"""GPU (CUDA library, through the C ABI) vs the FP64 oracle.

Populations are compared after up to 100 steps (the FP32 library against
the FP64 oracle from the same seeded start):

* relative 1e-6 on populations, as the relative L2 error of the field:
      ||f_gpu - f_ref||_2 / ||f_ref||_2 <= 1e-6;
* element by element, every node and direction:
      |f_gpu - f_ref| <= 3e-6 * max |f_ref|
      |f_gpu - f_ref| / max(|f_ref|, w_a rho_v) <= 1e-5.
  The element bounds come from the arithmetic: with exact arithmetic and only
  the FP32 storage rounding, the first measure already reaches 6.5e-7 after
  100 steps on a rough channel (a static interface node rounds the same way
  every step, so the errors add up rather than cancel), and the FP32
  collision multiplies that by about 2 at high-force interface nodes. The
  largest values measured over these cases on a GB300 are 2.2e-7 (L2),
  1.4e-6 (field-relative) and 5.3e-6 (self-relative); each case prints its
  three measures (pytest -s).
Every case also checks the observables (mass, flux Q of Eq. 11, momentum).
"""
import numpy as np
import pytest

import oracle
from paper_0708_4182_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
TOL_L2 = 1e-6      # relative L2 over the population field
TOL_FIELD = 3e-6   # per element, relative to the field's maximum
TOL_ELEM = 1e-5    # per element, relative to itself (vapor-scale floor)


@pytest.fixture(scope="module")
def lbm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0708_4182_gb300 import lbm as L
    L.load()
    return L


def pop_err(f_gpu, f_ref, mask, rho_v=wl.RHO_V):
    """(field-relative max, per-population max, relative L2) over fluid nodes."""
    fl = mask == 0
    d = np.abs(f_gpu - f_ref)[:, fl]
    r = np.abs(f_ref)[:, fl]
    field = float(d.max() / r.max())
    elem = float((d / np.maximum(r, W[:, None] * rho_v)).max())
    l2 = float(np.sqrt((d ** 2).sum() / (r ** 2).sum()))
    return field, elem, l2


def assert_pops(f_gpu, f_ref, mask):
    import os
    field, elem, l2 = pop_err(f_gpu, f_ref, mask)
    # the measured values, for the record (shown with pytest -s)
    print(f"\npopulation error [{os.environ.get('PYTEST_CURRENT_TEST', '?').split(' ')[0]}]: "
          f"rel_l2={l2:.3e} field_max={field:.3e} self_max={elem:.3e}")
    assert l2 <= TOL_L2 and field <= TOL_FIELD and elem <= TOL_ELEM, (l2, field, elem)
    assert np.all(f_gpu[:, mask == 1] == 0)


def run_both(lbm, mask, rho, params, steps, ux=0.0, uy=0.0, **lat_kw):
    ny, nx = mask.shape
    p = oracle.Params(nx, ny, **params)
    f0 = oracle.equilibrium(p, mask, rho, ux, uy)
    f_ref = oracle.step(p, mask, f0, steps)
    lat = lbm.Lattice(nx, ny, **params, **lat_kw)
    lat.set_geometry(mask)
    lat.set_rho_u(rho, ux, uy)
    lat.step(steps)
    return p, f_ref, lat


def check_obs(lat, p, mask, f_ref, rel=1e-6):
    o = lat.observables()
    r = oracle.observables(p, mask, f_ref)
    rho, jx, jy, t = oracle.forces(p, mask, f_ref)
    fx, fy = t[0::2].sum(0), t[1::2].sum(0)
    fl = mask == 0
    assert o["nonfinite"] == 0
    assert o["mass"] == pytest.approx(r["mass"], rel=rel)
    # j = sum_a f_a e_a cancels between populations of size ~rho, and
    # u = (j + F/2)/rho cancels again at interfaces (j ~ -F/2 at rest): a
    # node's u carries an error of a few 1e-7 (rho + |j| + |F|/2)/rho after
    # 100 FP32 steps, and Q and P sum these per-node errors
    mx = rho[fl] + np.abs(jx[fl]) + 0.5 * np.abs(fx[fl])
    my = rho[fl] + np.abs(jy[fl]) + 0.5 * np.abs(fy[fl])
    assert abs(o["flux_Q"] - r["flux_Q"]) <= 2e-6 * (mx / rho[fl]).sum() / p.nx
    assert abs(o["mom_x"] - r["mom_x"]) <= 2e-6 * mx.sum()
    assert abs(o["mom_y"] - r["mom_y"]) <= 2e-6 * my.sum()
    assert o["max_u"] == pytest.approx(r["max_u"], rel=1e-4)
    assert o["min_rho"] == pytest.approx(r["min_rho"], rel=1e-5)
    assert o["step"] == lat.time


@pytest.mark.parametrize("f_elec", wl.DROPLET_F_LEVELS)
def test_droplet_128x64_populations_100_steps(lbm, f_elec):
    w = wl.droplet_128x64(f_elec)
    p, f_ref, lat = run_both(lbm, w.mask, w.rho, w.params, 100)
    assert_pops(lat.populations(), f_ref, w.mask)
    check_obs(lat, p, w.mask, f_ref)


@pytest.mark.parametrize("level", [0, 9, 15])
def test_rough_channel_populations_100_steps(lbm, level):
    w = wl.rough_channel(nx=300, ny=48, amp=6, level=level, seed=5, body_fx=1e-5)
    p, f_ref, lat = run_both(lbm, w.mask, w.rho, w.params, 100)
    assert_pops(lat.populations(), f_ref, w.mask)
    check_obs(lat, p, w.mask, f_ref)


def test_rough_channel_1024x128_populations(lbm):
    """The rough-wall channel workload at its full size (1024 x 128, amp 8)."""
    w = wl.rough_channel(level=12)
    p, f_ref, lat = run_both(lbm, w.mask, w.rho, w.params, 100)
    assert_pops(lat.populations(), f_ref, w.mask)
    check_obs(lat, p, w.mask, f_ref)


def _blob_field(nx, ny, mask, seed):
    rng = np.random.default_rng(seed)
    cx, cy = rng.uniform(0, nx), rng.uniform(0, ny)
    rho = wl.droplet_field(nx, ny, [(cx, cy)], 0.3 * min(nx, ny) + 1.0, mask=mask)
    return rho


RAGGED = [
    # nx, ny, walls, tile_rows : strips of 256 columns and segments of tile_rows
    # rows with ragged ends, a single CTA, a single column, a single row
    (5, 4, False, 0),
    (1, 9, True, 0),
    (37, 11, True, 4),
    (254, 13, True, 8),
    (255, 20, True, 0),
    (509, 17, True, 4),
    (600, 1, False, 0),
    (131, 70, True, 64),
]


@pytest.mark.parametrize("layout", [1, 2])
@pytest.mark.parametrize("nx,ny,walls,tile_rows", RAGGED)
def test_ragged_and_tiny_domains(lbm, nx, ny, walls, tile_rows, layout):
    """Both thread layouts of the step kernel (pairs, one node per thread)
    against the oracle."""
    mask = np.zeros((ny, nx), np.uint8)
    if walls and ny >= 3:
        mask[0] = mask[-1] = 1
        if nx >= 8 and ny >= 8:
            mask[ny // 2:ny // 2 + 2, nx // 3:nx // 3 + 3] = 1  # an interior block
    rho = _blob_field(nx, ny, mask, nx * 1000 + ny)
    params = dict(wl.PAPER, tau=1.0, f_elec=0.2, body_fx=1e-5, body_fy=-2e-6)
    p, f_ref, lat = run_both(lbm, mask, rho, params, 40, tile_rows=tile_rows, layout=layout)
    assert_pops(lat.populations(), f_ref, mask)
    check_obs(lat, p, mask, f_ref)


@pytest.mark.parametrize("storage", [0, 1])
@pytest.mark.parametrize("tau", [1.0, 0.9])
def test_layouts_give_identical_populations(lbm, storage, tau):
    """The pair layout and the one-node layout of the 32-bit forms store the
    same bits (both are written with explicit roundings, operation for
    operation), on a rough channel with the electric force and ragged strips
    (520 columns), with tau = 1 and tau != 1; the fused observables agree and
    the per-node fields are identical."""
    w = wl.rough_channel(nx=520, ny=90, amp=6, level=9, seed=5, body_fx=1e-5)
    params = dict(w.params, tau=tau, storage=storage)
    pops, fields, obs = [], [], []
    for layout in (1, 2):
        lat = lbm.Lattice(w.nx, w.ny, **params, layout=layout, obs_every=7, tile_rows=8)
        lat.set_geometry(w.mask)
        lat.set_rho_u(w.rho)
        lat.step(42)
        pops.append(lat.populations())
        fields.append(lat.fields())
        obs.append(lat.obs_latest())
    assert np.array_equal(pops[0], pops[1])
    for a, b in zip(fields[0], fields[1]):
        assert np.array_equal(a, b)
    assert obs[0]["step"] == obs[1]["step"] == 35  # state 35, reduced by the step from it
    for k in ("max_u", "min_rho", "nonfinite"):
        assert obs[0][k] == obs[1][k], k
    for k in ("mass", "flux_Q", "mom_x", "mom_y"):
        assert obs[0][k] == pytest.approx(obs[1][k], rel=1e-12, abs=1e-15), k


def test_printed_green_convention_and_tau(lbm):
    """The other Green-function convention and tau != 1 (weaker G so that the
    printed weights are stable)."""
    w = wl.droplet_128x64(0.15)
    params = dict(w.params, G=-0.26, G_wall=-0.07, tau=0.95, green=oracle.GREEN_PRINTED)
    p, f_ref, lat = run_both(lbm, w.mask, w.rho, params, 100)
    assert_pops(lat.populations(), f_ref, w.mask)


def test_tiling_is_bitwise_invariant_and_deterministic(lbm):
    w = wl.rough_channel(nx=520, ny=90, amp=6, level=7, seed=3, body_fx=1e-5)
    outs = []
    for tr in (4, 8, 64, 4):
        lat = lbm.Lattice(w.nx, w.ny, **w.params, tile_rows=tr)
        lat.set_geometry(w.mask)
        lat.set_rho_u(w.rho)
        lat.step(30)
        outs.append(lat.populations())
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])


def test_fields_match_oracle(lbm):
    w = wl.droplet_128x64(0.25)
    p, f_ref, lat = run_both(lbm, w.mask, w.rho, w.params, 100)
    rho_g, ux_g, uy_g = lat.fields()
    rho_r, ux_r, uy_r = oracle.fields(p, w.mask, f_ref)
    np.testing.assert_allclose(rho_g, rho_r, rtol=2e-6, atol=0)
    umax = np.abs(np.r_[ux_r.ravel(), uy_r.ravel()]).max()
    assert np.abs(ux_g - ux_r).max() <= 1e-5 * umax
    assert np.abs(uy_g - uy_r).max() <= 1e-5 * umax


def test_ux_profile_matches_oracle(lbm):
    """LBM_UX_PROFILE: the x-averaged u_x(y) of a rough channel against the
    oracle's fields; summed over y it is the flux Q; the read-back leaves
    the state intact (stepping on still matches the oracle)."""
    w = wl.rough_channel(nx=256, ny=64, amp=6, level=10, seed=3, body_fx=1e-5)
    p, f_ref, lat = run_both(lbm, w.mask, w.rho, w.params, 100)
    prof = lat.ux_profile()
    _, ux, _ = oracle.fields(p, w.mask, f_ref)
    ref = np.where(w.mask == 0, ux, 0.0).mean(axis=1)
    assert prof.shape == (w.ny,)
    assert np.abs(prof - ref).max() <= 1e-5 * np.abs(ux).max()
    assert np.all(prof[0] == 0.0) and np.all(prof[-1] == 0.0)  # wall rows
    q = lat.observables()["flux_Q"]
    assert prof.sum() == pytest.approx(q, rel=1e-9, abs=1e-12)
    lat.step(50)
    assert_pops(lat.populations(), oracle.step(p, w.mask, f_ref, 50), w.mask)


def test_physical_velocity_state_matches_oracle(lbm):
    """LBM_RHO_U_PHYS: the state built from (rho, u), u the physical
    velocity, equals the oracle's equilibrium_physical populations, reads
    back as (rho, u) and steps like the oracle."""
    w = wl.rough_channel(nx=200, ny=48, amp=6, level=15, seed=4, body_fx=1e-5)
    p = oracle.Params(w.nx, w.ny, **w.params)
    f = oracle.step(p, w.mask, oracle.equilibrium(p, w.mask, w.rho, 0, 0), 200)
    rho, ux, uy = oracle.fields(p, w.mask, f)
    f_phys = oracle.equilibrium_physical(p, w.mask, rho, ux, uy)
    lat = lbm.Lattice(w.nx, w.ny, **w.params)
    lat.set_geometry(w.mask)
    lat.set_rho_u(rho, ux, uy, physical=True)
    assert_pops(lat.populations(), f_phys, w.mask)
    r2, u2, v2 = lat.fields()
    _, jx, jy, t = oracle.forces(p, w.mask, f_phys)
    fl = w.mask == 0
    scale = (rho + np.abs(jx) + np.abs(jy) + 0.5 * (np.abs(t[0::2].sum(0)) + np.abs(t[1::2].sum(0))))[fl] / rho[fl]
    np.testing.assert_allclose(r2[fl], rho[fl], rtol=2e-6)
    assert np.all(np.abs(u2[fl] - ux[fl]) <= 2e-6 * scale)
    assert np.all(np.abs(v2[fl] - uy[fl]) <= 2e-6 * scale)
    # the plain (rho, u) state differs by the F/2 shift at interfaces
    lat_plain = lbm.Lattice(w.nx, w.ny, **w.params)
    lat_plain.set_geometry(w.mask)
    lat_plain.set_rho_u(rho, ux, uy)
    assert np.abs(lat_plain.fields()[2] - uy)[fl].max() > 1e3 * np.abs(v2 - uy)[fl].max()
    lat.step(100)
    assert_pops(lat.populations(), oracle.step(p, w.mask, f_phys, 100), w.mask)


def test_population_round_trip_and_resume(lbm):
    """set/get of populations is exact in FP32, and a run resumed from a
    checkpoint is bitwise identical to an uninterrupted one."""
    w = wl.rough_channel(nx=300, ny=48, amp=6, level=15, seed=9, body_fx=1e-5)
    p = oracle.Params(w.nx, w.ny, **w.params)
    f0 = oracle.step(p, w.mask, oracle.equilibrium(p, w.mask, w.rho, 0, 0), 20)
    lat = lbm.Lattice(w.nx, w.ny, **w.params)
    lat.set_geometry(w.mask)
    lat.set_populations(f0)
    back = lat.populations()
    assert np.array_equal(back, f0.astype(np.float32).astype(np.float64))
    # uninterrupted 60 steps
    lat.step(60)
    ref = lat.populations()
    # 25 steps, checkpoint, fresh context, 35 steps
    lat2 = lbm.Lattice(w.nx, w.ny, **w.params)
    lat2.set_geometry(w.mask)
    lat2.set_populations(f0)
    lat2.step(25)
    ck = lat2.populations()
    lat3 = lbm.Lattice(w.nx, w.ny, **w.params)
    lat3.set_geometry(w.mask)
    lat3.set_populations(ck)
    lat3.step(35)
    assert np.array_equal(lat3.populations(), ref)
    # populations set from the oracle also step like the oracle
    assert_pops(ref, oracle.step(p, w.mask, f0, 60), w.mask)


def test_fused_observables_match_separate_pass(lbm):
    w = wl.droplet_128x64(0.125)
    lat = lbm.Lattice(w.nx, w.ny, **w.params, obs_every=10)
    lat.set_geometry(w.mask)
    lat.set_rho_u(w.rho)
    o0 = lat.observables()
    lat.step(1)
    f = lat.obs_latest()
    assert f["step"] == 0
    for k in ("mass", "flux_Q", "mom_x", "mom_y", "max_u", "min_rho"):
        assert f[k] == pytest.approx(o0[k], rel=1e-6, abs=1e-9)
    lat.step(24)
    assert lat.obs_latest()["step"] == 20
    o25 = lat.observables()
    assert o25["step"] == 25
    assert o25["mass"] == pytest.approx(o0["mass"], rel=1e-6)


@pytest.mark.parametrize("obs_every", [0, 37, 100])
def test_graph_stepping_equals_single_steps(lbm, obs_every):
    """lbm_step replays runs of 32 steps as a CUDA graph, stopping the graph
    windows at fused-observables steps: one call of 523 steps equals 523
    calls of one step bitwise, at any obs_every, and the latest fused record
    is that of the last observed step."""
    w = wl.rough_channel(nx=256, ny=64, amp=6, level=12, seed=2, body_fx=1e-5)
    runs = []
    for chunks in ([523], [1] * 523, [5, 64, 33, 421]):
        lat = lbm.Lattice(w.nx, w.ny, obs_every=obs_every, **w.params)
        lat.set_geometry(w.mask)
        lat.set_rho_u(w.rho)
        for n in chunks:
            lat.step(n)
        assert lat.time == 523
        runs.append((lat.populations(), lat.obs_latest() if obs_every else None))
    for pops, rec in runs[1:]:
        assert np.array_equal(pops, runs[0][0])
        if obs_every:
            assert rec["step"] == (522 // obs_every) * obs_every
            assert rec == runs[0][1]


def test_device_buffers(lbm):
    import torch
    w = wl.droplet_128x64(0.0625)
    lat = lbm.Lattice(w.nx, w.ny, **w.params)
    lat.set_geometry(torch.as_tensor(w.mask, device="cuda"))
    lat.set_rho_u(torch.as_tensor(w.rho, device="cuda"))
    lat.step(10)
    dev = lat.populations_device().cpu().numpy()
    assert np.array_equal(dev, lat.populations())


def test_nonfinite_reported(lbm):
    w = wl.droplet_128x64(0.0)
    p = oracle.Params(w.nx, w.ny, **w.params)
    f = oracle.equilibrium(p, w.mask, w.rho, 0, 0)
    f[2, 30, 40] = np.nan
    lat = lbm.Lattice(w.nx, w.ny, **w.params)
    lat.set_geometry(w.mask)
    lat.set_populations(f)
    with pytest.raises(lbm.LbmError) as e:
        lat.observables()
    assert e.value.status == lbm.LBM_ENAN
    o = lat.observables(check_finite=False)
    assert o["nonfinite"] >= 1


def test_error_paths(lbm):
    import torch
    p = lbm.make_params(64, 32)
    nbytes = lbm.lbm_workspace_bytes(p)
    assert nbytes > 0
    assert lbm.lbm_workspace_bytes(lbm.make_params(64, 32, tau=0.5)) == 0
    assert lbm.lbm_workspace_bytes(lbm.make_params(0, 32)) == 0
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_create(p, ws.data_ptr(), nbytes - 1, s)
    assert e.value.status == lbm.LBM_ENOMEM
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_create(lbm.make_params(64, 32, green=7), ws.data_ptr(), nbytes, s)
    assert e.value.status == lbm.LBM_EINVAL
    ctx = lbm.lbm_create(p, ws.data_ptr(), nbytes, s)
    try:
        with pytest.raises(lbm.LbmError) as e:
            lbm.lbm_step(ctx, 1)
        assert e.value.status == lbm.LBM_ESTATE
        mask = np.zeros((32, 64), np.uint8)
        lbm.lbm_set_geometry(ctx, mask.ctypes.data, False)
        with pytest.raises(lbm.LbmError) as e:
            lbm.lbm_step(ctx, 1)
        assert e.value.status == lbm.LBM_ESTATE
        with pytest.raises(lbm.LbmError) as e:
            lbm.lbm_set_field(ctx, 7, mask.ctypes.data, False)
        assert e.value.status == lbm.LBM_EINVAL
        assert "unknown field" in lbm.lbm_last_error(ctx)
        with pytest.raises(lbm.LbmError) as e:
            lbm.lbm_obs_latest(ctx)
        assert e.value.status == lbm.LBM_ESTATE
    finally:
        lbm.lbm_destroy(ctx)
    assert lbm.lbm_status_string(lbm.LBM_ENAN) == "LBM_ENAN"


def test_full_size_sampled_parity(lbm):
    """16384 x 4096 rough channel with the droplet row, in the benchmark's
    launch configuration. A node's state after k steps depends only on the
    state within Chebyshev distance 2k, so the oracle, run on a periodic crop
    with a halo of 2k+2 around a sample window, reproduces the window
    exactly; crops are cut from the generated inputs, never from GPU output."""
    import torch
    k = 3
    w = wl.droplet_row_channel()
    lat = lbm.Lattice(w.nx, w.ny, **w.params, obs_every=100)
    lat.set_geometry(w.mask)
    lat.set_rho_u(w.rho)
    m0 = lat.observables()["mass"]
    lat.step(k)
    dev = lat.populations_device()
    h, s = 2 * k + 2, 16
    rng = np.random.default_rng(0)
    windows = [(1, 60), (w.ny - 1 - s, 5000), (w.ny // 2, w.nx - 8), (3, 0)]
    windows += [(int(rng.integers(0, w.ny)), int(rng.integers(0, w.nx))) for _ in range(8)]
    for (y0, x0) in windows:
        ys = np.arange(y0 - h, y0 + s + h) % w.ny
        xs = np.arange(x0 - h, x0 + s + h) % w.nx
        mask = np.ascontiguousarray(w.mask[np.ix_(ys, xs)])
        rho = w.rho[np.ix_(ys, xs)]
        p = oracle.Params(len(xs), len(ys), **w.params)
        f_ref = oracle.step(p, mask, oracle.equilibrium(p, mask, rho, 0, 0), k)[:, h:h + s, h:h + s]
        yi = torch.as_tensor(ys[h:h + s], device=dev.device)
        xi = torch.as_tensor(xs[h:h + s], device=dev.device)
        f_gpu = dev[:, yi][:, :, xi].cpu().numpy()
        assert_pops(f_gpu, f_ref, mask[h:h + s, h:h + s])
    del dev
    # properties at full size: mass conserved (FP64 reduction of FP32 state)
    lat.step(97)
    o = lat.observables()
    assert o["nonfinite"] == 0
    assert abs(o["mass"] - m0) <= 1e-6 * m0
    assert lat.obs_latest()["step"] == 0


def test_bounded_wait_times_out_and_context_survives(lbm):
    """The device-side timeout path, without a fault: a kernel waits on an
    mbarrier phase that nothing completes, gives up after its bounded number
    of polls, and the host reads LBM_ETIMEOUT; the context then steps on and
    matches an undisturbed run bitwise."""
    w = wl.droplet_128x64(0.125)
    lat = lbm.Lattice(w.nx, w.ny, **w.params)
    lat.set_geometry(w.mask)
    lat.set_rho_u(w.rho)
    lat.step(10)
    assert lbm.lbm_selftest_timeout(lat.ctx) == lbm.LBM_ETIMEOUT
    assert "gave up" in lbm.lbm_last_error(lat.ctx)
    lat.step(40)
    assert lat.observables()["nonfinite"] == 0
    ref = lbm.Lattice(w.nx, w.ny, **w.params)
    ref.set_geometry(w.mask)
    ref.set_rho_u(w.rho)
    ref.step(50)
    assert np.array_equal(lat.populations(), ref.populations())


@pytest.mark.gpu
def test_obs_latest_async_matches_synchronous_read(lbm):
    """The enqueued copy of the latest fused record (no synchronisation in
    the call) equals the record the synchronising read returns."""
    import ctypes
    import torch
    w = wl.droplet_128x64(0.125)
    lat = lbm.Lattice(w.nx, w.ny, obs_every=1, **w.params)
    lat.set_geometry(w.mask)
    lat.set_rho_u(w.rho)
    buf = torch.empty(ctypes.sizeof(lbm.lbm_obs), dtype=torch.uint8).pin_memory()
    for _ in range(3):
        lat.step(7)
        lbm.lbm_obs_latest_async(lat.ctx, buf.data_ptr())
        torch.cuda.synchronize()
        assert lbm.obs_from_buffer(buf.data_ptr()) == lbm.lbm_obs_latest(lat.ctx)
    lat.close()


@pytest.mark.parametrize("storage", [0, 1, 2, 3])
def test_density_only_setup_equals_rest_equilibrium(lbm, storage):
    """LBM_RHO (a fluid at rest from its density alone) gives the state that
    LBM_RHO_U gives with zero velocity, bit for bit, in every storage form,
    before and after stepping."""
    w = wl.rough_channel(nx=256, ny=48, amp=6, level=9, seed=5, body_fx=1e-5)
    a = lbm.Lattice(w.nx, w.ny, storage=storage, **w.params)
    b = lbm.Lattice(w.nx, w.ny, storage=storage, **w.params)
    for lat in (a, b):
        lat.set_geometry(w.mask)
    a.set_rho_u(w.rho)
    b.set_rho(w.rho)
    assert np.array_equal(a.populations(), b.populations())
    a.step(7)
    b.step(7)
    assert np.array_equal(a.populations(), b.populations())


@pytest.mark.parametrize("storage", [0, 1, 2, 3])
def test_fp32_density_setup(lbm, storage):
    """lbm_set_density_f32 (FP32 set-up arithmetic) against LBM_RHO (FP64,
    rounded once) on a rough channel with a droplet row: the populations
    agree to FP32 rounding (relative to the field's maximum: 2e-7 in the
    32-bit forms; the 16-bit forms round both to the same deviations but
    for the rare value on a rounding boundary), from host and device input,
    and 40 steps from it stay within the oracle tolerances."""
    import torch
    w = wl.droplet_row_channel(nx=512, ny=96, amp=6, seed=2, radius=12.0, pitch=96, body_fx=1e-5, f_elec=0.125)
    rho32 = np.where(w.mask == 0, w.rho, 0.0).astype(np.float32)
    ref = lbm.Lattice(w.nx, w.ny, **dict(w.params, storage=storage))
    ref.set_geometry(w.mask)
    ref.set_rho(rho32.astype(np.float64))
    fr = ref.populations()
    fl = w.mask == 0
    scale = np.abs(fr[:, fl]).max()
    for device in (False, True):
        lat = lbm.Lattice(w.nx, w.ny, **dict(w.params, storage=storage))
        lat.set_geometry(w.mask)
        lat.set_density_f32(torch.from_numpy(rho32).cuda() if device else rho32)
        f = lat.populations()
        err = np.abs(f - fr)[:, fl].max() / scale
        bound = 2e-7 if storage < 2 else 2e-3
        assert err <= bound, (device, err)
        assert np.all(f[:, ~fl] == 0)
        if not device:
            lat.step(40)
            p = oracle.Params(w.nx, w.ny, **w.params)
            f_ref = oracle.step(p, w.mask, oracle.equilibrium(p, w.mask, rho32.astype(np.float64), 0, 0), 40)
            if storage < 2:
                assert_pops(lat.populations(), f_ref, w.mask)
        lat.close()
    ref.close()


def test_unit_normal_reading_matches_oracle(lbm):
    """The electric force along the unit face normal (LBM_NORMAL_UNIT) on a
    rough channel full of liquid, so that conductive liquid fills the
    concave step corners, where the two readings differ (with vapor in the
    grooves no corner is conductive and they coincide): populations after
    100 steps within the gates, and different from the per-face reading's."""
    w = wl.rough_channel(nx=300, ny=48, amp=6, level=15, seed=5, body_fx=1e-5, fill=1.0)
    params = dict(w.params, normal=1)
    p = oracle.Params(w.nx, w.ny, **params)
    f_ref = oracle.step(p, w.mask, oracle.equilibrium(p, w.mask, w.rho, 0, 0), 100)
    lat = lbm.Lattice(w.nx, w.ny, **params)
    lat.set_geometry(w.mask)
    lat.set_rho_u(w.rho)
    lat.step(100)
    assert_pops(lat.populations(), f_ref, w.mask)
    check_obs(lat, p, w.mask, f_ref)
    p_faces = oracle.Params(w.nx, w.ny, **w.params)
    f_faces = oracle.step(p_faces, w.mask, oracle.equilibrium(p_faces, w.mask, w.rho, 0, 0), 100)
    assert pop_err(f_faces, f_ref, w.mask)[0] > 1e-3
