"""The allocation-free observables entry point against the context one.

lbm_observables_noalloc serves callers that cannot allocate device memory
when they need observables: processes whose device memory budget is spent,
and monitoring or checkpoint tools that hold a state in their own buffers and
must not touch the application's allocator. It keeps its scratch in a static
device array of the library instead of a workspace. These tests call it
through the C ABI on the populations and mask of a running context, twice in
a row (the second call reuses the scratch the first one left behind), and
compare its output with lbm_observables on the same state, within the
tolerance the other observables tests use. They also check that a call
leaves the device's free memory unchanged, and run a domain at the size limit
(16,777,216 nodes), where every one of the 1024 partial slots is written.
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


def test_noalloc_allocates_nothing(lbm):
    """Free device memory is the same before and after a call (after a first
    call has loaded everything the library needs)."""
    import torch
    w = wl.rough_channel(nx=300, ny=48, amp=6, level=3, seed=2, body_fx=1e-5)
    lat = lbm.Lattice(w.nx, w.ny, **w.params)
    lat.set_geometry(w.mask)
    lat.set_rho_u(w.rho)
    lat.step(10)
    pops = lat.populations_device()
    d_mask = torch.as_tensor(w.mask, device="cuda")
    args = (lat.params, pops.data_ptr(), d_mask.data_ptr(), lat.time, lat.stream.cuda_stream)
    lbm.lbm_observables_noalloc(*args)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    reserved0 = torch.cuda.memory_reserved()
    for _ in range(3):
        lbm.lbm_observables_noalloc(*args)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_reserved() == reserved0


def test_noalloc_at_the_size_limit(lbm):
    """4096 x 4096 = 16,777,216 nodes: the largest accepted domain, whose
    1024 CTAs fill every partial slot of the static array."""
    import torch
    w = wl.droplet_row_channel(nx=4096, ny=4096, amp=6, seed=3, f_elec=0.15)
    lat = lbm.Lattice(w.nx, w.ny, **w.params)
    lat.set_geometry(w.mask)
    lat.set_rho_u(w.rho)
    lat.step(6)
    pops = lat.populations_device()
    d_mask = torch.as_tensor(w.mask, device="cuda")
    for _ in range(2):
        ref = lat.observables()
        got = lbm.lbm_observables_noalloc(lat.params, pops.data_ptr(), d_mask.data_ptr(), lat.time,
                                          lat.stream.cuda_stream)
        assert got["nonfinite"] == ref["nonfinite"] == 0
        for k in FIELDS:
            assert got[k] == pytest.approx(ref[k], rel=1e-6, abs=1e-9), k
    del pops
