"""Pins of the U-Net CPU reference (oracle/unet_oracle.py).

* its autograd gradients agree with central finite differences (FP64);
* the circular x padding makes the network equivariant to shifts along x
  by multiples of the coarsest stride (8 columns);
* the layer shapes give the stated parameter count (4 levels, 32 base
  channels, 3 inputs, 3 outputs).
"""
import torch

from oracle import unet_oracle as U


def tiny_params(scale=1.0, seed=0):
    g = torch.Generator().manual_seed(seed)
    p = {}
    for name, (co, ci, k) in U.shapes().items():
        std = scale * (2.0 / (ci * k * k)) ** 0.5
        p[name] = (torch.randn((co, ci, k, k), generator=g, dtype=torch.float64) * std,
                   torch.randn(co, generator=g, dtype=torch.float64) * 0.01)
    return p


def test_parameter_count():
    n = sum(co * ci * k * k + co for co, ci, k in U.shapes().values())
    # weights: encoder 9 (32*3 + 32*32 + 64*32 + 64*64 + 128*64 + 128*128 + 256*128 + 256*256)
    # = 1,171,296; decoder 9 (128*384 + 128*128 + 64*192 + 64*64 + 32*96 + 32*32) = 774,144;
    # head 3*32 = 96; biases 960 + 448 + 3 = 1,411
    assert n == 1171296 + 774144 + 96 + 1411


def test_translation_equivariance_along_x():
    p = tiny_params()
    g = torch.Generator().manual_seed(1)
    x = torch.randn((1, 3, 32, 64), generator=g, dtype=torch.float64)
    y = U.forward(p, x)
    ys = U.forward(p, torch.roll(x, 8, dims=3))
    assert torch.allclose(torch.roll(y, 8, dims=3), ys, rtol=1e-10, atol=1e-12)


def test_gradients_match_finite_differences():
    p = tiny_params(seed=2)
    g = torch.Generator().manual_seed(3)
    x = torch.randn((1, 3, 32, 64), generator=g, dtype=torch.float64)
    t = torch.randn((1, 3, 32, 64), generator=g, dtype=torch.float64)
    wc = torch.tensor([1.0, 0.5, 2.0], dtype=torch.float64)
    _, grads = U.loss_and_grads(p, x, t, wc)
    for name, idx in [("e0a", (3, 1, 0, 2)), ("e3b", (5, 7, 1, 1)), ("d1a", (2, 100, 2, 0)),
                      ("d0b", (31, 4, 1, 2)), ("head", (2, 17, 0, 0))]:
        w, b = p[name]
        h = 1e-6
        wp = w.clone(); wp[idx] += h
        wm = w.clone(); wm[idx] -= h
        fp = U.loss({**p, name: (wp, b)}, x, t, wc).item()
        fm = U.loss({**p, name: (wm, b)}, x, t, wc).item()
        fd = (fp - fm) / (2 * h)
        assert abs(fd - grads[name][0][idx].item()) <= 1e-6 * max(1.0, abs(fd)), name
