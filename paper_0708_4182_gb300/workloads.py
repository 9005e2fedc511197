"""Seeded synthetic inputs: wall masks and initial density/velocity fields.

This module holds no arithmetic of the lattice Boltzmann method itself. It
builds the inputs both the CUDA library and the CPU oracle start from:

* rough-wall channel masks: rectangular steps of width a, height b and
  centre distance p on the top and bottom walls of a periodic channel (the
  rough-wall channel sketch of the paper; a, b, p are not given there, so they
  are drawn from a seeded SplitMix64 stream);
* initial density fields: a sessile droplet or a row of droplets on the bottom
  wall, or a central liquid slab, with tanh edges between the liquid and vapor
  plateau densities;
* the parameter sets of the five workloads (droplet 128x64, rough channel
  1024x128, 256 batched channels, 16384x4096 precision study, 256x64 learned
  warm-start tiles).

Random draws use SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) so that the
same seed gives the same geometry in any language.
"""
from __future__ import annotations

import dataclasses

import numpy as np

# Liquid and vapor plateau densities of this model at G = -0.52, rho0 = 1 with
# the Martys-Chen link weights (flat-interface equilibrium, rounded). They only
# shape initial conditions; the tests check that the oracle's own plateau
# lies within 1% of them.
RHO_L = 2.805
RHO_V = 0.0631

_MASK64 = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 generator (64-bit state, golden-ratio increment)."""

    def __init__(self, seed: int):
        self.state = seed & _MASK64

    def next(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
        return z ^ (z >> 31)

    def randint(self, lo: int, hi: int) -> int:
        """Integer uniform on [lo, hi] (inclusive)."""
        return lo + self.next() % (hi - lo + 1)

    def uniform(self) -> float:
        """Double uniform on [0, 1) from the top 53 bits."""
        return (self.next() >> 11) * (1.0 / (1 << 53))


def wall_profile(nx: int, amp: int, rng: SplitMix64, width=(4, 16), gap=(4, 32)) -> np.ndarray:
    """Step heights along one wall: repeat (gap, width a, height b) until the
    next element would pass nx; the leftover columns join the first gap across
    the periodic seam. Heights are b in [0, amp]."""
    h = np.zeros(nx, dtype=np.int32)
    x = 0
    while True:
        g = rng.randint(*gap)
        a = rng.randint(*width)
        b = rng.randint(0, amp) if amp > 0 else 0
        if x + g + a > nx:
            break
        h[x + g:x + g + a] = b
        x += g + a
    return h


def channel_mask(nx: int, ny: int, amp: int = 0, seed: int = 0, width=(4, 16),
                 gap=(4, 32)) -> np.ndarray:
    """Solid mask (uint8, shape (ny, nx), 1 = solid) of a periodic channel:
    rows 0 and ny-1 are walls; each wall carries seeded steps of height up to
    ``amp`` (bottom and top use independent streams derived from ``seed``)."""
    if ny < 3:
        raise ValueError("a channel needs ny >= 3")
    mask = np.zeros((ny, nx), dtype=np.uint8)
    mask[0, :] = 1
    mask[ny - 1, :] = 1
    if amp > 0:
        if 2 * amp + 3 > ny:
            raise ValueError("roughness amplitude too large for this height")
        seeder = SplitMix64(seed)
        bottom = wall_profile(nx, amp, SplitMix64(seeder.next()), width, gap)
        top = wall_profile(nx, amp, SplitMix64(seeder.next()), width, gap)
        ys = np.arange(ny)[:, None]
        mask[(ys >= 1) & (ys <= bottom[None, :])] = 1
        mask[(ys <= ny - 2) & (ys >= ny - 1 - top[None, :])] = 1
    return mask


def tanh_profile(dist: np.ndarray, rho_in: float, rho_out: float, width: float) -> np.ndarray:
    """rho_in inside (dist < 0), rho_out outside, tanh edge of given width."""
    return 0.5 * (rho_in + rho_out) - 0.5 * (rho_in - rho_out) * np.tanh(2.0 * dist / width)


def droplet_field(nx: int, ny: int, centres, radius: float, rho_l=RHO_L, rho_v=RHO_V,
                  width: float = 4.0, mask=None) -> np.ndarray:
    """Density of one or more 2D droplets (discs of the given radius centred at
    ``centres`` = [(cx, cy), ...]) in vapor; zero on solid nodes."""
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    dist = np.full((ny, nx), np.inf)
    for cx, cy in centres:
        dx = np.abs(x - cx)
        dx = np.minimum(dx, nx - dx)  # periodic in x
        dist = np.minimum(dist, np.sqrt(dx * dx + (y - cy) ** 2) - radius)
    rho = tanh_profile(dist, rho_l, rho_v, width)
    if mask is not None:
        rho = np.where(mask != 0, 0.0, rho)
    return rho


def slab_field(nx: int, ny: int, fill: float = 0.5, rho_l=RHO_L, rho_v=RHO_V,
               width: float = 4.0, mask=None, axis: int = 0) -> np.ndarray:
    """A liquid slab centred in the domain, occupying ``fill`` of the height
    (axis 0) or length (axis 1), vapor elsewhere; zero on solid nodes."""
    n = ny if axis == 0 else nx
    c = 0.5 * (n - 1)
    half = 0.5 * fill * (n - 2)
    s = np.arange(n, dtype=np.float64)
    prof = tanh_profile(np.abs(s - c) - half, rho_l, rho_v, width)
    rho = np.broadcast_to(prof[:, None] if axis == 0 else prof[None, :], (ny, nx)).copy()
    if mask is not None:
        rho = np.where(mask != 0, 0.0, rho)
    return rho


@dataclasses.dataclass
class Workload:
    """One synthetic domain: parameters, wall mask and initial (rho, ux, uy)."""
    name: str
    nx: int
    ny: int
    mask: np.ndarray
    rho: np.ndarray
    params: dict
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def ux(self):
        return np.zeros((self.ny, self.nx))

    @property
    def uy(self):
        return np.zeros((self.ny, self.nx))


# Parameters the paper fixes (droplet run): G = -0.52, w = -0.14, rho0 = 1,
# rho_c = 1; the workloads use tau = 1.0.
PAPER = dict(G=-0.52, G_wall=-0.14, rho0=1.0, rho_c=1.0)

# Electric-force amplitudes: 0 up to the paper's largest value, 0.25.
F_ELEC_MAX = 0.25
DROPLET_F_LEVELS = (0.0, 0.0625, 0.125, 0.1875, 0.25)


def f_level(level: int) -> float:
    """Electric-force amplitude of sweep level 0..15 (0 .. 0.25)."""
    return F_ELEC_MAX * level / 15.0


def droplet_128x64(f_elec: float = 0.0, radius: float = 20.0) -> Workload:
    """Sessile droplet of radius 20 on the smooth bottom wall of a periodic
    128x64 box with walls at y = 0 and y = 63 (tau = 1)."""
    nx, ny = 128, 64
    mask = channel_mask(nx, ny)
    rho = droplet_field(nx, ny, [(nx / 2, 0.5)], radius, mask=mask)
    return Workload("droplet_128x64", nx, ny, mask, rho,
                    dict(PAPER, tau=1.0, f_elec=f_elec, body_fx=0.0, body_fy=0.0))


def rough_channel(nx=1024, ny=128, amp=8, level=0, seed=0, fill=None, body_fx=1e-6) -> Workload:
    """Rough-wall channel filled with electrolyte, driven by a uniform body
    force; electric force at sweep ``level``. By default the liquid fills the
    channel up to the crests of the tallest roughness elements and the grooves
    between elements hold vapor, so the electrolyte touches the walls (the
    electric force acts only on liquid next to a wall)."""
    mask = channel_mask(nx, ny, amp, seed)
    if fill is None:
        fill = max(0.1, 1.0 - 2.0 * (amp + 1) / (ny - 2))
    rho = slab_field(nx, ny, fill, mask=mask)
    return Workload(f"rough_channel_{nx}x{ny}", nx, ny, mask, rho,
                    dict(PAPER, tau=1.0, f_elec=f_level(level), body_fx=body_fx, body_fy=0.0),
                    dict(amp=amp, level=level, fill=fill, seed=seed))


def droplet_row_channel(nx=16384, ny=4096, amp=6, seed=0, radius=20.0, pitch=128,
                        body_fx=1e-6, f_elec=0.0) -> Workload:
    """Large rough-wall channel (vapor) with a row of sessile droplets of the
    given radius and pitch on the bottom wall; body-force driven."""
    mask = channel_mask(nx, ny, amp, seed)
    centres = [(pitch / 2 + k * pitch, 0.5) for k in range(nx // pitch)]
    rho = droplet_row_density(nx, ny, centres, radius, mask)
    return Workload(f"droplet_row_channel_{nx}x{ny}", nx, ny, mask, rho,
                    dict(PAPER, tau=1.0, f_elec=f_elec, body_fx=body_fx, body_fy=0.0))


def droplet_row_density(nx, ny, centres, radius, mask, width=4.0):
    """Row-of-droplets density built band by band (only rows near the bottom
    wall hold liquid), so very large domains stay cheap to generate."""
    rho = np.full((ny, nx), RHO_V)
    top = int(min(ny, max(cy for _, cy in centres) + radius + 4 * width + 2))
    band = droplet_field(nx, top, centres, radius, width=width)
    rho[:top] = band
    return np.where(mask != 0, 0.0, rho)


def stepped_channel_mask(nx: int, width: int, a: int, b: int, pitch: int) -> np.ndarray:
    """Solid mask of the paper's rough-wall channel sketch: a periodic channel
    of `width` fluid rows between two solid rows, both walls carrying
    rectangular steps of width a and height b whose centres are `pitch` apart
    (the same x positions on both walls); nx must be a multiple of pitch."""
    if nx % pitch or a >= pitch or 2 * b + 1 > width:
        raise ValueError("steps do not fit the channel")
    ny = width + 2
    mask = np.zeros((ny, nx), dtype=np.uint8)
    mask[0, :] = 1
    mask[ny - 1, :] = 1
    x = np.arange(nx)
    on = ((x - pitch // 2 + a // 2) % pitch) < a  # step centred at pitch/2 of each period
    mask[1:b + 1, on] = 1
    mask[ny - 1 - b:ny - 1, on] = 1
    return mask


def paper_channel(width: int, f_elec: float, nx: int = 256, a: int = 8, b: int = 8, pitch: int = 32,
                  body_fx: float = 8e-6, perturb: float = 1e-3, seed: int = 11) -> Workload:
    """The paper's electrowetting channel runs: rough-wall channel of width 160
    or 80 under a rightward body force 8e-6, electric force 0, 0.15 or 0.25.
    The paper gives neither the step sizes a, b, p nor the length; these are
    chosen (a = b = 8, p = 32, length 256). Liquid fills the channel up to the
    step crests, vapor fills the grooves between steps. The channel is mirror
    symmetric, and a symmetric start stays symmetric in a deterministic
    update; each node's density is therefore scaled by 1 + perturb * xi, xi
    uniform on [-1, 1) from a SplitMix64 stream (seed), so that an unstable
    symmetric state (the paper's narrow channel at strong f) can break."""
    mask = stepped_channel_mask(nx, width, a, b, pitch)
    ny = width + 2
    fill = 1.0 - 2.0 * (b + 1) / (ny - 2)
    rho = slab_field(nx, ny, fill, mask=mask)
    if perturb:
        rng = SplitMix64(seed)
        xi = np.array([2.0 * rng.uniform() - 1.0 for _ in range(nx * ny)]).reshape(ny, nx)
        rho = rho * (1.0 + perturb * xi)
    return Workload(f"paper_channel_w{width}", nx, ny, mask, rho,
                    dict(PAPER, tau=1.0, f_elec=f_elec, body_fx=body_fx, body_fy=0.0),
                    dict(width=width, a=a, b=b, pitch=pitch, fill=fill))


def batched_channels(count=256, seed=0):
    """Sizes and levels of the batched sweep: width 32-256, length 512-2048,
    roughness amplitude 0-8 and electric-force level 0-15, from one seed."""
    rng = SplitMix64(seed)
    out = []
    for k in range(count):
        ny = rng.randint(32, 256)
        nx = rng.randint(512, 2048)
        amp = min(rng.randint(0, 8), (ny - 3) // 2)
        level = rng.randint(0, 15)
        out.append(dict(nx=nx, ny=ny, amp=amp, level=level, seed=rng.next()))
    return out


def warm_start_channels(count, seed=0, nx=256, ny=64, body_fx=1e-5):
    """Channels of the warm-start surrogate: nx x ny rough channels of the
    rough-channel recipe with roughness amplitude 0-8, electric-force level
    0-15 and a fill fraction drawn between the crest fill (liquid up to the
    tallest roughness elements) and halfway from there to a full channel,
    from one seed. A lower fill leaves the liquid floating on vapor layers,
    where the body force accelerates it without bound."""
    rng = SplitMix64(seed)
    out = []
    for _ in range(count):
        amp = rng.randint(0, 8)
        level = rng.randint(0, 15)
        crest = 1.0 - 2.0 * (amp + 1) / (ny - 2)
        fill = crest + 0.5 * (1.0 - crest) * rng.uniform()
        out.append(rough_channel(nx=nx, ny=ny, amp=amp, level=level, seed=rng.next(), fill=fill,
                                 body_fx=body_fx))
    return out


def smooth_channels(count, seed=0, nx=256, ny=64, body_fx=1e-5):
    """Flat-wall channels (the smooth-channel geometry) of varying height:
    bottom and top walls 1 + U{0..8} rows thick, electric-force level 0-15,
    a centred liquid slab whose fill fraction of the free gap is drawn
    between the crest fill 1 - 2/gap and 1, from one seed."""
    rng = SplitMix64(seed)
    out = []
    for _ in range(count):
        tb, tt = rng.randint(0, 8), rng.randint(0, 8)
        level = rng.randint(0, 15)
        mask = np.zeros((ny, nx), dtype=np.uint8)
        mask[:1 + tb] = 1
        mask[ny - 1 - tt:] = 1
        gap = ny - 2 - tb - tt
        crest = 1.0 - 2.0 / gap
        fill = crest + (1.0 - crest) * rng.uniform()
        ys = np.arange(ny, dtype=np.float64)
        centre = 0.5 * ((1 + tb) + (ny - 2 - tt))
        prof = tanh_profile(np.abs(ys - centre) - 0.5 * fill * gap, RHO_L, RHO_V, 4.0)
        rho = np.where(mask != 0, 0.0, np.broadcast_to(prof[:, None], (ny, nx)))
        out.append(Workload(f"smooth_channel_{nx}x{ny}", nx, ny, mask, rho,
                            dict(PAPER, tau=1.0, f_elec=f_level(level), body_fx=body_fx, body_fy=0.0),
                            dict(amp=0, level=level, fill=fill, seed=seed, walls=(tb, tt))))
    return out
