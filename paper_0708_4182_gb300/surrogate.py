"""Warm-start surrogate: a 4-level U-Net (32 base channels) on 256 x 64 tiles.

Input planes: wall mask, electric-force level / 15, fill fraction. Output:
steady density and velocity (normalised), used through lbm_set_field
(LBM_RHO_U) as the initial state of a lattice Boltzmann run that then runs
on to convergence. Training data are steady states the LBM itself produces.

All arithmetic runs in the hand-written kernels of libunet_bf16 (BF16
storage, FP32 accumulation, FP32 master weights with Adam); this module only
sequences layers and owns the buffers (torch CUDA tensors used as memory).
Architecture and padding are those of the CPU reference network used by the
tests: encoder levels with (32, 64, 128, 256) channels, two 3x3
convolutions + ReLU each, 2x2 average pooling; decoder levels upsample
(nearest), concatenate [upsampled, skip] and apply two 3x3 convolutions +
ReLU; a 1x1 head gives 3 channels.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

C = (32, 64, 128, 256)
IN_CH, OUT_CH = 3, 3

_lib = None


def load_unet():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.UNET_LIB):
        from .lbm import LbmUnavailable
        raise LbmUnavailable(f"{_build.UNET_LIB} is not built; run __graft_entry__.build()")
    lib = ctypes.CDLL(_build.UNET_LIB)
    vp, L, I, F, D = ctypes.c_void_p, ctypes.c_long, ctypes.c_int, ctypes.c_float, ctypes.c_double
    sig = {
        "unet_conv3x3_fwd": [vp, I, L, vp, vp, vp, I, L, I, I, I, I, vp],
        "unet_conv3x3_bwd_data": [vp, I, L, vp, vp, I, L, I, I, I, vp],
        "unet_conv3x3_bwd_weight": [vp, I, L, vp, I, L, vp, vp, I, I, I, vp],
        "unet_head_fwd": [vp, I, L, vp, vp, vp, I, I, I, vp],
        "unet_head_bwd": [vp, I, L, vp, vp, I, I, I, vp, L, vp, vp, vp],
        "unet_pool2_fwd": [vp, L, vp, L, I, I, I, I, vp],
        "unet_pool2_bwd": [vp, L, vp, L, I, I, I, I, I, vp],
        "unet_up2_fwd": [vp, L, vp, L, I, I, I, I, vp],
        "unet_up2_bwd": [vp, L, vp, L, I, I, I, I, vp],
        "unet_relu_bwd": [vp, L, vp, L, I, I, vp],
        "unet_mse": [vp, vp, vp, I, I, L, vp, vp, vp],
        "unet_adam": [vp, vp, vp, vp, vp, L, F, F, F, F, I, F, vp],
        "unet_f32_to_bf16": [vp, vp, L, vp],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes, fn.restype = args, ctypes.c_int
    _lib = lib
    return lib


def _call(fn, *args):
    rc = fn(*args)
    if rc != 0:
        raise RuntimeError(f"{fn.__name__} failed with {rc}")


def layer_shapes() -> dict:
    s = {}
    cin = IN_CH
    for l, c in enumerate(C):
        s[f"e{l}a"] = (c, cin, 3)
        s[f"e{l}b"] = (c, c, 3)
        cin = c
    for l in (2, 1, 0):
        s[f"d{l}a"] = (C[l], C[l + 1] + C[l], 3)
        s[f"d{l}b"] = (C[l], C[l], 3)
    s["head"] = (OUT_CH, C[0], 1)
    return s


class View:
    """A channel range of an NCHW buffer: (tensor, channel offset, channels)."""

    def __init__(self, t, c0, c):
        self.t, self.c0, self.c = t, c0, c

    @property
    def ptr(self):
        n, ct, h, w = self.t.shape
        return self.t.data_ptr() + self.c0 * h * w * self.t.element_size()

    @property
    def bs(self):
        n, ct, h, w = self.t.shape
        return ct * h * w


class UNet:
    """Parameters, optimizer state and activation buffers for batch size B."""

    def __init__(self, batch=16, height=64, width=256, seed=0, stream=None):
        import torch
        self.torch = torch
        self.lib = load_unet()
        self.B, self.H, self.W = batch, height, width
        if height % 32 or width % 256:
            raise ValueError("height must be a multiple of 32 and width of 256")
        self.dev = "cuda"
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.s = ctypes.c_void_p(self.stream.cuda_stream)
        g = torch.Generator().manual_seed(seed)
        self.params = {}
        for name, (co, ci, k) in layer_shapes().items():
            std = (2.0 / (ci * k * k)) ** 0.5
            wm = (torch.randn((co, ci, k, k), generator=g, dtype=torch.float64) * std).float().to(self.dev)
            self.params[name] = self._param(wm, torch.zeros(co, device=self.dev))
        self.step_count = 0
        self.norm = dict(rho_mean=1.5, rho_std=1.0, u_scale=1e-3)
        self._alloc(batch)

    def _param(self, wm, bm):
        t = self.torch
        bf = t.empty_like(wm, dtype=t.bfloat16)
        p = dict(w=wm.contiguous(), b=bm.contiguous(), wb=bf, gw=t.zeros_like(wm), gb=t.zeros_like(bm),
                 mw=t.zeros_like(wm), vw=t.zeros_like(wm), mb=t.zeros_like(bm), vb=t.zeros_like(bm))
        _call(self.lib.unet_f32_to_bf16, ctypes.c_void_p(p["w"].data_ptr()), ctypes.c_void_p(bf.data_ptr()),
              p["w"].numel(), self.s)
        return p

    def set_weights(self, weights: dict):
        """Load FP32 weights/biases {name: (w, b)} (e.g. to match a reference)."""
        for name, (w, b) in weights.items():
            p = self.params[name]
            p["w"].copy_(self.torch.as_tensor(w, dtype=self.torch.float32))
            p["b"].copy_(self.torch.as_tensor(b, dtype=self.torch.float32))
            _call(self.lib.unet_f32_to_bf16, ctypes.c_void_p(p["w"].data_ptr()),
                  ctypes.c_void_p(p["wb"].data_ptr()), p["w"].numel(), self.s)

    def weights(self) -> dict:
        return {k: (p["w"].detach().cpu().numpy(), p["b"].detach().cpu().numpy()) for k, p in self.params.items()}

    def _alloc(self, B):
        t = self.torch
        H, W = self.H, self.W
        bf = dict(dtype=t.bfloat16, device=self.dev)
        hw = [(H >> l, W >> l) for l in range(4)]
        self.x0 = t.zeros((B, IN_CH, H, W), **bf)
        self.A = [t.zeros((B, C[l], *hw[l]), **bf) for l in range(4)]
        self.B3 = t.zeros((B, C[3], *hw[3]), **bf)
        self.cat = [t.zeros((B, C[l + 1] + C[l], *hw[l]), **bf) for l in range(3)]
        self.P = [t.zeros((B, C[l], *hw[l + 1]), **bf) for l in range(3)]
        self.DA = [t.zeros((B, C[l], *hw[l]), **bf) for l in range(3)]
        self.DB = [t.zeros((B, C[l], *hw[l]), **bf) for l in range(3)]
        self.out = t.zeros((B, OUT_CH, H, W), dtype=t.float32, device=self.dev)
        # gradients of the activations
        self.gA = [t.zeros_like(a) for a in self.A]
        self.gB3 = t.zeros_like(self.B3)
        self.gcat = [t.zeros_like(c) for c in self.cat]
        self.gP = [t.zeros_like(p) for p in self.P]
        self.gDA = [t.zeros_like(a) for a in self.DA]
        self.gDB = [t.zeros_like(a) for a in self.DB]
        self.gout = t.zeros_like(self.out)
        self.loss_acc = t.zeros(1, dtype=t.float64, device=self.dev)
        self.batch = B

    # -------------------------------------------------------------- layers
    def _conv(self, name, x: View, y: View, h, w, relu=True):
        p = self.params[name]
        co, ci, _ = layer_shapes()[name]
        _call(self.lib.unet_conv3x3_fwd, ctypes.c_void_p(x.ptr), ci, x.bs, ctypes.c_void_p(p["wb"].data_ptr()),
              ctypes.c_void_p(p["b"].data_ptr()), ctypes.c_void_p(y.ptr), co, y.bs, self.batch, h, w,
              1 if relu else 0, self.s)

    def _conv_bwd(self, name, x: View, y: View, gy: View, gx: View | None, h, w):
        """Through relu(conv(x)): gy *= (y > 0); accumulate weight/bias grads;
        gx = conv^T(gy) if gx is given."""
        p = self.params[name]
        co, ci, _ = layer_shapes()[name]
        lib, n = self.lib, self.batch
        _call(lib.unet_relu_bwd, ctypes.c_void_p(y.ptr), y.bs, ctypes.c_void_p(gy.ptr), gy.bs, co * h * w, n, self.s)
        _call(lib.unet_conv3x3_bwd_weight, ctypes.c_void_p(x.ptr), ci, x.bs, ctypes.c_void_p(gy.ptr), co, gy.bs,
              ctypes.c_void_p(p["gw"].data_ptr()), ctypes.c_void_p(p["gb"].data_ptr()), n, h, w, self.s)
        if gx is not None:
            _call(lib.unet_conv3x3_bwd_data, ctypes.c_void_p(gy.ptr), co, gy.bs, ctypes.c_void_p(p["wb"].data_ptr()),
                  ctypes.c_void_p(gx.ptr), ci, gx.bs, n, h, w, self.s)

    def forward(self, x_planes):
        """x_planes: float tensor [B, 3, H, W] on the device -> self.out (FP32)."""
        lib, n, s = self.lib, self.batch, self.s
        H, W = self.H, self.W
        xs = x_planes.contiguous().float()
        _call(lib.unet_f32_to_bf16, ctypes.c_void_p(xs.data_ptr()), ctypes.c_void_p(self.x0.data_ptr()),
              xs.numel(), s)
        h = View(self.x0, 0, IN_CH)
        for l in range(4):
            hh, ww = H >> l, W >> l
            a = View(self.A[l], 0, C[l])
            self._conv(f"e{l}a", h, a, hh, ww)
            if l < 3:
                skip = View(self.cat[l], C[l + 1], C[l])
                self._conv(f"e{l}b", a, skip, hh, ww)
                _call(lib.unet_pool2_fwd, ctypes.c_void_p(skip.ptr), skip.bs, ctypes.c_void_p(self.P[l].data_ptr()),
                      C[l] * (hh // 2) * (ww // 2), C[l], n, hh, ww, s)
                h = View(self.P[l], 0, C[l])
            else:
                self._conv("e3b", a, View(self.B3, 0, C[3]), hh, ww)
        lower = View(self.B3, 0, C[3])
        for l in (2, 1, 0):
            hh, ww = H >> l, W >> l
            up = View(self.cat[l], 0, C[l + 1])
            _call(lib.unet_up2_fwd, ctypes.c_void_p(lower.ptr), lower.bs, ctypes.c_void_p(up.ptr), up.bs,
                  C[l + 1], n, hh // 2, ww // 2, s)
            self._conv(f"d{l}a", View(self.cat[l], 0, C[l + 1] + C[l]), View(self.DA[l], 0, C[l]), hh, ww)
            self._conv(f"d{l}b", View(self.DA[l], 0, C[l]), View(self.DB[l], 0, C[l]), hh, ww)
            lower = View(self.DB[l], 0, C[l])
        hp = self.params["head"]
        _call(lib.unet_head_fwd, ctypes.c_void_p(lower.ptr), C[0], lower.bs, ctypes.c_void_p(hp["wb"].data_ptr()),
              ctypes.c_void_p(hp["b"].data_ptr()), ctypes.c_void_p(self.out.data_ptr()), OUT_CH, n, H * W, s)
        return self.out

    def loss_backward(self, target, wc):
        """MSE against target [B, 3, H, W] (FP32) with channel weights wc;
        fills every parameter gradient (zeroed first); returns the loss."""
        t, lib, n, s = self.torch, self.lib, self.batch, self.s
        H, W = self.H, self.W
        for p in self.params.values():
            p["gw"].zero_()
            p["gb"].zero_()
        self.loss_acc.zero_()
        tg = target.contiguous().float()
        wct = t.as_tensor(wc, dtype=t.float32, device=self.dev)
        _call(lib.unet_mse, ctypes.c_void_p(self.out.data_ptr()), ctypes.c_void_p(tg.data_ptr()),
              ctypes.c_void_p(wct.data_ptr()), OUT_CH, H * W, self.out.numel(),
              ctypes.c_void_p(self.gout.data_ptr()), ctypes.c_void_p(self.loss_acc.data_ptr()), s)
        hp = self.params["head"]
        gdb0 = View(self.gDB[0], 0, C[0])
        _call(lib.unet_head_bwd, ctypes.c_void_p(self.DB[0].data_ptr()), C[0], C[0] * H * W,
              ctypes.c_void_p(hp["wb"].data_ptr()), ctypes.c_void_p(self.gout.data_ptr()), OUT_CH, n, H * W,
              ctypes.c_void_p(gdb0.ptr), gdb0.bs, ctypes.c_void_p(hp["gw"].data_ptr()),
              ctypes.c_void_p(hp["gb"].data_ptr()), s)
        gup = None
        for l in (0, 1, 2):
            hh, ww = H >> l, W >> l
            if gup is not None:
                # gradient of level l's decoder output arrives through the upsampling
                _call(lib.unet_up2_bwd, ctypes.c_void_p(gup.ptr), gup.bs, ctypes.c_void_p(self.gDB[l].data_ptr()),
                      C[l] * hh * ww, C[l], n, hh, ww, s)
            self._conv_bwd(f"d{l}b", View(self.DA[l], 0, C[l]), View(self.DB[l], 0, C[l]),
                           View(self.gDB[l], 0, C[l]), View(self.gDA[l], 0, C[l]), hh, ww)
            self._conv_bwd(f"d{l}a", View(self.cat[l], 0, C[l + 1] + C[l]), View(self.DA[l], 0, C[l]),
                           View(self.gDA[l], 0, C[l]), View(self.gcat[l], 0, C[l + 1] + C[l]), hh, ww)
            gup = View(self.gcat[l], 0, C[l + 1])  # towards the level below (coarser)
        # bottleneck: gradient of B3 through the level-2 upsampling
        hh, ww = H >> 3, W >> 3
        _call(lib.unet_up2_bwd, ctypes.c_void_p(gup.ptr), gup.bs, ctypes.c_void_p(self.gB3.data_ptr()),
              C[3] * hh * ww, C[3], n, hh, ww, s)
        self._conv_bwd("e3b", View(self.A[3], 0, C[3]), View(self.B3, 0, C[3]), View(self.gB3, 0, C[3]),
                       View(self.gA[3], 0, C[3]), hh, ww)
        self._conv_bwd("e3a", View(self.P[2], 0, C[2]), View(self.A[3], 0, C[3]), View(self.gA[3], 0, C[3]),
                       View(self.gP[2], 0, C[2]), hh, ww)
        for l in (2, 1, 0):
            hh, ww = H >> l, W >> l
            gskip = View(self.gcat[l], C[l + 1], C[l])
            _call(lib.unet_pool2_bwd, ctypes.c_void_p(self.gP[l].data_ptr()), C[l] * (hh // 2) * (ww // 2),
                  ctypes.c_void_p(gskip.ptr), gskip.bs, C[l], n, hh, ww, 1, s)
            self._conv_bwd(f"e{l}b", View(self.A[l], 0, C[l]), View(self.cat[l], C[l + 1], C[l]), gskip,
                           View(self.gA[l], 0, C[l]), hh, ww)
            below = View(self.x0, 0, IN_CH) if l == 0 else View(self.P[l - 1], 0, C[l - 1])
            self._conv_bwd(f"e{l}a", below, View(self.A[l], 0, C[l]), View(self.gA[l], 0, C[l]),
                           None if l == 0 else View(self.gP[l - 1], 0, C[l - 1]), hh, ww)
        return float(self.loss_acc.item())

    def adam(self, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=0.0):
        self.step_count += 1
        for p in self.params.values():
            _call(self.lib.unet_adam, ctypes.c_void_p(p["w"].data_ptr()), ctypes.c_void_p(p["wb"].data_ptr()),
                  ctypes.c_void_p(p["gw"].data_ptr()), ctypes.c_void_p(p["mw"].data_ptr()),
                  ctypes.c_void_p(p["vw"].data_ptr()), p["w"].numel(), lr, beta1, beta2, eps, self.step_count,
                  weight_decay, self.s)
            _call(self.lib.unet_adam, ctypes.c_void_p(p["b"].data_ptr()), None, ctypes.c_void_p(p["gb"].data_ptr()),
                  ctypes.c_void_p(p["mb"].data_ptr()), ctypes.c_void_p(p["vb"].data_ptr()), p["b"].numel(), lr,
                  beta1, beta2, eps, self.step_count, 0.0, self.s)

    # -------------------------------------------------------- data mapping
    def planes(self, masks, levels, fills):
        """Input planes [B, 3, H, W]: mask, level/15, fill."""
        t = self.torch
        m = t.as_tensor(np.asarray(masks), dtype=t.float32, device=self.dev)
        lv = t.as_tensor(np.asarray(levels, dtype=np.float32) / 15.0, device=self.dev)[:, None, None]
        fl = t.as_tensor(np.asarray(fills, dtype=np.float32), device=self.dev)[:, None, None]
        return t.stack([m, lv.expand_as(m), fl.expand_as(m)], dim=1)

    def encode_targets(self, rho, ux, uy):
        t, nm = self.torch, self.norm
        r = (t.as_tensor(rho, dtype=t.float32, device=self.dev) - nm["rho_mean"]) / nm["rho_std"]
        return t.stack([r, t.as_tensor(ux, dtype=t.float32, device=self.dev) / nm["u_scale"],
                        t.as_tensor(uy, dtype=t.float32, device=self.dev) / nm["u_scale"]], dim=1)

    def decode(self, out):
        nm = self.norm
        rho = out[:, 0] * nm["rho_std"] + nm["rho_mean"]
        return rho, out[:, 1] * nm["u_scale"], out[:, 2] * nm["u_scale"]
