"""Plain PyTorch CPU reference of the warm-start U-Net (FP64).

TEST INFRASTRUCTURE ONLY: the tests compare the CUDA kernels' outputs and
gradients with this module; the CUDA library never uses it.

Network (4 levels, 32 base channels), written out layer by layer:
  encoder level l = 0..3 with C = (32, 64, 128, 256) channels:
      h = relu(conv3(h, e{l}a)); h = relu(conv3(h, e{l}b));
      for l < 3 keep h as skip l and halve the resolution by 2x2 averaging;
  decoder level l = 2, 1, 0:
      h = nearest 2x upsampling of h; h = concat(h, skip l) along channels;
      h = relu(conv3(h, d{l}a)); h = relu(conv3(h, d{l}b));
  output: 1x1 convolution "head" to 3 channels (density, u_x, u_y).
conv3 pads circularly in x (the channels are periodic along the flow) and
with zeros in y (walls). Loss: mean over all outputs of wc[c] (y - t)^2.
Parameters are a dict name -> (weight, bias) of torch tensors with the
shapes of ``shapes()``; gradients come from torch.autograd.
"""
from __future__ import annotations

import torch
import torch.nn.functional as F

C = (32, 64, 128, 256)
IN_CH, OUT_CH = 3, 3


def shapes(in_ch: int = IN_CH) -> dict:
    """name -> (out_channels, in_channels, kernel size) for every layer."""
    s = {}
    cin = in_ch
    for l, c in enumerate(C):
        s[f"e{l}a"] = (c, cin, 3)
        s[f"e{l}b"] = (c, c, 3)
        cin = c
    for l in (2, 1, 0):
        s[f"d{l}a"] = (C[l], C[l + 1] + C[l], 3)
        s[f"d{l}b"] = (C[l], C[l], 3)
    s["head"] = (OUT_CH, C[0], 1)
    return s


def conv3(x, w, b):
    x = F.pad(x, (1, 1, 0, 0), mode="circular")
    x = F.pad(x, (0, 0, 1, 1))
    return F.conv2d(x, w, b)


def forward(params: dict, x: torch.Tensor) -> torch.Tensor:
    skips = []
    h = x
    for l in range(4):
        h = torch.relu(conv3(h, *params[f"e{l}a"]))
        h = torch.relu(conv3(h, *params[f"e{l}b"]))
        if l < 3:
            skips.append(h)
            h = F.avg_pool2d(h, 2)
    for l in (2, 1, 0):
        h = F.interpolate(h, scale_factor=2, mode="nearest")
        h = torch.cat([h, skips[l]], dim=1)
        h = torch.relu(conv3(h, *params[f"d{l}a"]))
        h = torch.relu(conv3(h, *params[f"d{l}b"]))
    w, b = params["head"]
    return F.conv2d(h, w, b)


def loss(params: dict, x: torch.Tensor, target: torch.Tensor, wc: torch.Tensor) -> torch.Tensor:
    y = forward(params, x)
    return (wc[None, :, None, None] * (y - target) ** 2).mean()


def loss_and_grads(params: dict, x, target, wc):
    """Loss and d(loss)/d(weight), d(loss)/d(bias) for every layer (FP64)."""
    p = {k: (w.detach().double().clone().requires_grad_(True), b.detach().double().clone().requires_grad_(True))
         for k, (w, b) in params.items()}
    out = loss(p, x.double(), target.double(), wc.double())
    out.backward()
    return out.item(), {k: (w.grad, b.grad) for k, (w, b) in p.items()}
