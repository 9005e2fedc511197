"""Host-side pins: the contact-angle measurement and the seeded inputs.

The contact-angle measurement is checked on synthetic circular caps whose
angle is known in closed form (cos theta = -(y_c - 1/2)/R for a circle of
radius R centred at height y_c above the wall plane y = 1/2). The geometry
generator is checked against the rough-wall recipe: solid wall rows, steps of
width 4-16 and height 0..amp separated by gaps of 4-32, reproducible from the
seed.
"""
import numpy as np
import pytest

from paper_0708_4182_gb300 import workloads as wl
from tests._analysis import cos_contact_angle


@pytest.mark.parametrize("yc,R", [(10.0, 15.0), (0.5, 18.0), (-6.0, 20.0), (4.0, 16.0)])
def test_contact_angle_of_circular_cap(yc, R):
    nx, ny = 128, 64
    mask = wl.channel_mask(nx, ny)
    rho = wl.droplet_field(nx, ny, [(64.0, yc)], R, mask=mask)
    c, (xc, ycf, Rf) = cos_contact_angle(rho, wl.RHO_L, wl.RHO_V, mask)
    assert c == pytest.approx(-(yc - 0.5) / R, abs=2e-3)
    assert xc == pytest.approx(64.0, abs=1e-6)


def test_splitmix64_reference_values():
    # first outputs for seed 1234567 (published test vector of SplitMix64)
    g = wl.SplitMix64(1234567)
    out = [g.next() for _ in range(3)]
    assert out == [6457827717110365317, 3203168211198807973, 9817491932198370423]


@pytest.mark.parametrize("nx,ny,amp,seed", [(1024, 128, 8, 0), (700, 60, 6, 3), (512, 32, 0, 1)])
def test_channel_mask_recipe(nx, ny, amp, seed):
    m = wl.channel_mask(nx, ny, amp, seed)
    assert m.dtype == np.uint8 and m.shape == (ny, nx)
    assert np.all(m[0] == 1) and np.all(m[-1] == 1)
    assert np.array_equal(m, wl.channel_mask(nx, ny, amp, seed))
    bottom = m[1:ny // 2].sum(0)
    top = m[ny // 2:-1].sum(0)
    for h in (bottom, top):
        assert h.min() >= 0 and h.max() <= amp
    # solid cells of each column are contiguous from the wall
    for x in range(nx):
        col = m[:, x]
        b, t = bottom[x], top[x]
        assert np.all(col[1:1 + b] == 1) and np.all(col[1 + b:ny - 1 - t] == 0)
    if amp > 0:
        rng = wl.SplitMix64(seed)
        prof = wl.wall_profile(nx, amp, wl.SplitMix64(rng.next()))
        assert np.array_equal(prof, bottom)
        # element widths in [4, 16]; the gaps between elements in [4, 32]
        # except the seam gap, which may absorb the leftover columns
        xs = np.nonzero(np.diff(np.r_[0, (prof > 0).astype(int)]))[0]
        assert len(xs) > 0


def test_wall_profile_elements():
    rng = wl.SplitMix64(99)
    nx = 4096
    h = np.full(nx, -1)
    x = 0
    gaps, widths = [], []
    # regenerate with the same stream and record the draws
    g = wl.SplitMix64(99)
    while True:
        gap, a, b = g.randint(4, 32), g.randint(4, 16), g.randint(0, 8)
        if x + gap + a > nx:
            break
        gaps.append(gap)
        widths.append(a)
        x += gap + a
    prof = wl.wall_profile(nx, 8, rng)
    assert min(gaps) >= 4 and max(gaps) <= 32
    assert min(widths) >= 4 and max(widths) <= 16
    assert prof.max() <= 8
    assert sum(gaps) + sum(widths) <= nx


def test_batched_channel_sizes():
    chans = wl.batched_channels(256, seed=0)
    assert len(chans) == 256
    for c in chans:
        assert 32 <= c["ny"] <= 256 and 512 <= c["nx"] <= 2048
        assert 0 <= c["amp"] <= 8 and 0 <= c["level"] <= 15
        assert 2 * c["amp"] + 3 <= c["ny"]
    assert chans == wl.batched_channels(256, seed=0)


def test_droplet_workload_shapes():
    w = wl.droplet_128x64(0.1)
    assert w.rho.shape == (64, 128) and w.mask.shape == (64, 128)
    assert np.all(w.rho[w.mask == 1] == 0)
    assert w.rho[1, 64] > 2.5 and w.rho[40, 10] < 0.1
    assert w.params["f_elec"] == 0.1 and w.params["tau"] == 1.0
    assert wl.f_level(15) == 0.25 and wl.f_level(0) == 0.0
