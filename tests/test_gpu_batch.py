"""Batched sweeps: many uneven domains advanced by one persistent launch.

The batch runs the same per-node arithmetic as a single domain, and the
result does not depend on the tiling, so every domain of a batch must be
bitwise identical to the same domain stepped alone, which is itself checked
against the FP64 oracle. Also covered: batched observables, the active set,
the tile-height autotuner and run-to-steady against the oracle's steady flux.
"""
import numpy as np
import pytest

import oracle
from paper_0708_4182_gb300 import workloads as wl
from tests.test_gpu_parity import assert_pops

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0708_4182_gb300 import lbm as L
    L.load()
    return L


def sweep_workloads(count=6, seed=11, storage=0):
    """A small sweep of uneven channels in the batched-sweep recipe."""
    out = []
    for k, ch in enumerate(wl.batched_channels(count, seed)):
        nx = max(64, ch["nx"] // 4 // 8 * 8)
        ny = max(2 * ch["amp"] + 8, ch["ny"] // 3)
        w = wl.rough_channel(nx=nx, ny=ny, amp=min(ch["amp"], (ny - 3) // 2), level=ch["level"],
                             seed=ch["seed"], body_fx=1e-5)
        out.append(w)
    return out


def specs_of(ws, storage=0):
    return [dict(nx=w.nx, ny=w.ny, storage=storage, **w.params) for w in ws]


@pytest.mark.parametrize("storage,layout", [(0, 0), (0, 1), (0, 2), (1, 0), (1, 1), (1, 2), (2, 0), (3, 0)])
def test_batch_equals_single_domain_runs(lbm, storage, layout):
    """Each domain of a batch equals the same domain stepped alone, bitwise;
    the batch's thread layout (automatic or forced) need not be the single
    domain's (automatic) one."""
    ws = sweep_workloads(storage=storage)
    b = lbm.Batch([dict(s, layout=layout) for s in specs_of(ws, storage)])
    b.set_tile_rows(16)
    for w, d in zip(ws, b.domains):
        d.set_geometry(w.mask)
        d.set_rho_u(w.rho)
    b.step(37)  # odd: graph pairs plus one single launch
    for w, d in zip(ws, b.domains):
        lat = lbm.Lattice(w.nx, w.ny, storage=storage, **w.params)
        lat.set_geometry(w.mask)
        lat.set_rho_u(w.rho)
        lat.step(37)
        assert np.array_equal(d.populations(), lat.populations())
        assert d.time == 37
    obs = b.observables()
    for w, d, o in zip(ws, b.domains, obs):
        single = d.observables()
        for k in ("mass", "flux_Q", "mom_x", "mom_y", "max_u", "min_rho"):
            assert o[k] == pytest.approx(single[k], rel=1e-12, abs=1e-15), k
    b.close()


@pytest.mark.parametrize("storage,layout", [(0, 1), (0, 2), (2, 0)])
def test_batch_tiny_and_ragged_domains_equal_single_runs(lbm, storage, layout):
    """Tiny and ragged domains in one batch (an 8-column domain whose staged
    window wraps many times, a single row, strips with ragged ends): each
    equals the same domain stepped alone, bitwise."""
    from tests.test_gpu_parity import _blob_field
    shapes = [(8, 16), (24, 30), (248, 13), (600, 1), (264, 20)]
    params = dict(wl.PAPER, tau=1.0, f_elec=0.2, body_fx=1e-5, body_fy=-2e-6)
    cases = []
    for nx, ny in shapes:
        mask = np.zeros((ny, nx), np.uint8)
        if ny >= 3:
            mask[0] = mask[-1] = 1
        cases.append((mask, _blob_field(nx, ny, mask, nx * 1000 + ny)))
    b = lbm.Batch([dict(nx=m.shape[1], ny=m.shape[0], storage=storage, layout=layout, **params)
                   for m, _ in cases])
    b.set_tile_rows(8)
    for (m, rho), d in zip(cases, b.domains):
        d.set_geometry(m)
        d.set_rho_u(rho)
    b.step(21)
    for (m, rho), d in zip(cases, b.domains):
        lat = lbm.Lattice(m.shape[1], m.shape[0], storage=storage, **params)
        lat.set_geometry(m)
        lat.set_rho_u(rho)
        lat.step(21)
        assert np.array_equal(d.populations(), lat.populations()), m.shape
    b.close()


def test_batch_domain_matches_oracle(lbm):
    ws = sweep_workloads(4, seed=5)
    b = lbm.Batch(specs_of(ws))
    for w, d in zip(ws, b.domains):
        d.set_geometry(w.mask)
        d.set_rho_u(w.rho)
    b.step(60)
    for w, d in zip(ws, b.domains):
        p = oracle.Params(w.nx, w.ny, **w.params)
        f_ref = oracle.step(p, w.mask, oracle.equilibrium(p, w.mask, w.rho, 0, 0), 60)
        assert_pops(d.populations(), f_ref, w.mask)
    b.close()


def test_batch_active_set_and_autotune(lbm):
    ws = sweep_workloads(5, seed=3)
    b = lbm.Batch(specs_of(ws))
    for w, d in zip(ws, b.domains):
        d.set_geometry(w.mask)
        d.set_rho_u(w.rho)
    frozen = b.domains[2].populations()
    b.set_active([1, 1, 0, 1, 1])
    b.step(10)
    assert np.array_equal(b.domains[2].populations(), frozen)
    assert b.domains[2].time == 0 and b.domains[0].time == 10
    chosen, ms = b.autotune((8, 16, 32), steps=4)
    assert chosen in (8, 16, 32) and all(m > 0 for m in ms)
    assert b.tile_rows == chosen
    assert b.domains[0].time == 10 + 3 * 6 and b.domains[2].time == 0
    b.close()


def test_batch_autotune_grid_and_ctas_per_sm(lbm):
    """Tile height x CTAs per SM: every pair is timed, the fastest kept, and
    the result does not depend on the grid (bitwise equal populations)."""
    ws = sweep_workloads(4, seed=5)
    outs = []
    for ctas in (1, 3):
        b = lbm.Batch(specs_of(ws))
        for w, d in zip(ws, b.domains):
            d.set_geometry(w.mask)
            d.set_rho_u(w.rho)
        b.set_ctas_per_sm(ctas)
        assert b.ctas_per_sm == ctas
        b.step(9)
        outs.append([d.populations() for d in b.domains])
        if ctas == 3:
            rows, cts, table = b.autotune_grid((8, 32), (2, 3), steps=4)
            assert set(table) == {(8, 2), (32, 2), (8, 3), (32, 3)} and all(v > 0 for v in table.values())
            assert table[(rows, cts)] == min(table.values())
            assert b.tile_rows == rows and b.ctas_per_sm == cts
            probe = lbm.Batch(specs_of(ws))
            top = probe.ctas_per_sm  # the default: the most that fit
            probe.close()
            with pytest.raises(lbm.LbmError):
                b.set_ctas_per_sm(top + 1)
        b.close()
    for a, c in zip(*outs):
        assert np.array_equal(a, c)


def test_batch_run_to_steady_matches_oracle(lbm):
    """Three smooth channels at levels 0, 10, 15 in one batch (FP32
    deviation storage), each run to steady flux; the steady Q match the
    oracle's within 1e-4."""
    from tests.test_gpu_steady import oracle_steady_cached, smooth_channel
    ws = [smooth_channel(lv) for lv in (0, 10, 15)]
    b = lbm.Batch(specs_of(ws, storage=1))
    for w, d in zip(ws, b.domains):
        d.set_geometry(w.mask)
        d.set_rho_u(w.rho)
    steps, obs, ok = b.run_to_steady(1e-7, 1000, 80000)
    assert ok, steps
    for lv, o, st in zip((0, 10, 15), obs, steps):
        qr, tr = oracle_steady_cached(lv)
        assert o["flux_Q"] == pytest.approx(qr, rel=1e-4), (lv, o["flux_Q"], qr)
        assert 0 < st <= tr + 3000
    b.close()


def test_batch_rejects_mixed_storage(lbm):
    ws = sweep_workloads(2)
    sp = specs_of(ws)
    sp[1]["storage"] = 1
    with pytest.raises(lbm.LbmError):
        lbm.Batch(sp)


def test_batch_run_to_steady_drops_non_finite_domain(lbm):
    """A domain that turns non-finite (here: a NaN density planted in its
    initial field on the host) is dropped with steps -2; the others still
    run to steady flux, and the call reports LBM_ENAN."""
    from tests.test_gpu_steady import smooth_channel
    ws = [smooth_channel(0), smooth_channel(10)]
    b = lbm.Batch(specs_of(ws, storage=1))
    for w, d in zip(ws, b.domains):
        d.set_geometry(w.mask)
    rho = ws[0].rho.copy()
    rho[20, 64] = np.nan
    b.domains[0].set_rho_u(rho)
    b.domains[1].set_rho_u(ws[1].rho)
    steps, obs, ok = b.run_to_steady(1e-7, 1000, 80000)
    assert not ok
    assert steps[0] == -2 and obs[0]["nonfinite"] > 0
    assert steps[1] > 0 and np.isfinite(obs[1]["flux_Q"])
    assert "non-finite" in lbm._batch_lib().lbm_batch_last_error(b.handle).decode()
    b.close()
