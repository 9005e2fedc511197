"""The allocation-free observables entry point against the context one.

lbm_observables_noalloc serves callers that cannot allocate device memory
when they need observables: code running while a CUDA graph is captured,
processes whose device memory budget is spent, and tools that hold a state
in their own buffers. It keeps its scratch in a static device array of the
library instead of a workspace. These tests call it through the C ABI on the
populations and mask of a running context, twice in a row (the second call
reuses the scratch the first one left behind), and compare its output with
lbm_observables on the same state, within the tolerance the other
observables tests use.
"""
import numpy as np
import pytest

from paper_0708_4182_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

FIELDS = ("mass", "flux_Q", "mom_x", "mom_y", "max_u", "min_rho")


@pytest.fixture(scope="module")
def lbm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0708_4182_gb300 import lbm as L
    L.load()
    return L


def test_noalloc_matches_context_observables_twice(lbm):
    import torch
    w = wl.rough_channel(nx=300, ny=48, amp=6, level=12, seed=5, body_fx=1e-5)
    lat = lbm.Lattice(w.nx, w.ny, **w.params)
    lat.set_geometry(w.mask)
    lat.set_rho_u(w.rho)
    d_mask = torch.as_tensor(w.mask, device="cuda")
    for steps in (20, 35):
        lat.step(steps)
        ref = lat.observables()
        pops = lat.populations_device()
        got = lbm.lbm_observables_noalloc(lat.params, pops.data_ptr(), d_mask.data_ptr(), lat.time,
                                          lat.stream.cuda_stream)
        assert got["step"] == ref["step"] == lat.time
        assert got["nonfinite"] == ref["nonfinite"] == 0
        for k in FIELDS:
            assert got[k] == pytest.approx(ref[k], rel=1e-6, abs=1e-9), k


def test_noalloc_droplet_with_walls(lbm):
    import torch
    w = wl.droplet_128x64(0.25)
    lat = lbm.Lattice(w.nx, w.ny, **w.params)
    lat.set_geometry(w.mask)
    lat.set_rho_u(w.rho)
    lat.step(40)
    ref = lat.observables()
    pops = lat.populations_device()
    d_mask = torch.as_tensor(w.mask, device="cuda")
    got = lbm.lbm_observables_noalloc(lat.params, pops.data_ptr(), d_mask.data_ptr(), 7,
                                      lat.stream.cuda_stream)
    assert got["step"] == 7
    for k in FIELDS:
        assert got[k] == pytest.approx(ref[k], rel=1e-6, abs=1e-9), k


def test_noalloc_rejects_oversized_domain(lbm):
    p = lbm.make_params(8192, 4096)  # 33.5 M nodes, above the 16.8 M limit
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_observables_noalloc(p, 1 << 20, 1 << 20, 0, 0)
    assert e.value.status == lbm.LBM_EINVAL
    assert "exceeds the allocation-free limit" in str(e.value)
