"""Warm-start surrogate: a 4-level U-Net (32 base channels) on 256 x 64 tiles.

Input planes: wall mask, electric-force level / 15, fill fraction. Output:
steady density and velocity (normalised), used through lbm_set_field
(LBM_RHO_U_PHYS) as the initial state of a lattice Boltzmann run that then
runs on to convergence. Training data are steady states the LBM itself
produces.

All arithmetic runs in the hand-written kernels of libunet_bf16: 3x3
convolutions and their gradients on the tensor cores (tcgen05, BF16 operands,
FP32 accumulation), the rest as CUDA-core kernels; activations are BF16
channels-last, master weights and Adam moments FP32. This module only
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
IN_PAD = 16  # input channels as stored (the convolutions read 16 channels per step)

_lib = None


def load_unet():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.UNET_LIB):
        from .lbm import LbmUnavailable
        raise LbmUnavailable(f"{_build.UNET_LIB} is not built; run __graft_entry__.build()")
    lib = ctypes.CDLL(_build.UNET_LIB)
    vp, L, I, F = ctypes.c_void_p, ctypes.c_long, ctypes.c_int, ctypes.c_float
    sig = {
        "unet_conv_ntile": ([I], I),
        "unet_conv_pack_elems": ([I, I, I], ctypes.c_size_t),
        "unet_conv_pack": ([vp, I, I, I, vp, vp], I),
        "unet_conv_pack_many": ([vp, I, L, vp], I),
        "unet_conv3x3": ([vp, I, I, vp, vp, vp, I, I, I, I, I, I, vp], I),
        "unet_conv3x3_bwd_weight": ([vp, I, I, vp, I, I, vp, vp, I, I, I, vp], I),
        "unet_tc_error": ([vp, I], I),
        "unet_head_fwd": ([vp, I, I, vp, vp, vp, I, I, I, vp], I),
        "unet_head_bwd": ([vp, I, I, vp, vp, I, I, I, vp, I, vp, vp, vp], I),
        "unet_pool2_fwd": ([vp, I, vp, I, I, I, I, I, vp], I),
        "unet_pool2_bwd": ([vp, I, vp, I, I, I, I, I, I, vp], I),
        "unet_up2_fwd": ([vp, I, vp, I, I, I, I, I, vp], I),
        "unet_up2_bwd": ([vp, I, vp, I, I, I, I, I, vp], I),
        "unet_relu_bwd": ([vp, I, vp, I, I, L, vp, vp], I),
        "unet_input_nhwc": ([vp, I, I, I, vp, I, vp], I),
        "unet_mse": ([vp, vp, vp, I, I, L, vp, vp, vp], I),
        "unet_adam": ([vp, vp, vp, vp, vp, L, F, F, F, F, I, F, vp], I),
        "unet_adam_dev": ([vp, vp, vp, vp, vp, L, vp, F, F, F, F, vp], I),
        "unet_adam_hyper": ([vp, vp, I, F, F, vp], I),
        "unet_f32_to_bf16": ([vp, vp, L, vp], I),
        "unet_warm_fields": ([vp, I, I, vp, vp, F, F, F, ctypes.c_double, ctypes.c_double, vp, vp, vp], I),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes, fn.restype = args, res
    _lib = lib
    return lib


def _call(fn, *args):
    rc = fn(*args)
    if rc != 0:
        raise RuntimeError(f"{fn.__name__} failed with {rc}")


def layer_shapes(in_ch: int = IN_CH) -> dict:
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


class View:
    """A channel range of an NHWC buffer: (tensor, channel offset, channels)."""

    def __init__(self, t, c0, c):
        self.t, self.c0, self.c = t, c0, c

    @property
    def ptr(self):
        return ctypes.c_void_p(self.t.data_ptr() + self.c0 * self.t.element_size())

    @property
    def ct(self):
        return self.t.shape[-1]


class UNet:
    """Parameters, optimizer state and activation buffers for batch size B."""

    def __init__(self, batch=16, height=64, width=256, seed=0, stream=None, in_ch=IN_CH):
        import torch
        self.torch = torch
        self.lib = load_unet()
        self.B, self.H, self.W = batch, height, width
        if height % 32 or width % 256:
            raise ValueError("height must be a multiple of 32 and width of 256")
        if in_ch > IN_PAD:
            raise ValueError(f"at most {IN_PAD} input planes")
        self.in_ch = in_ch
        self.shapes = layer_shapes(in_ch)
        self.dev = "cuda"
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.s = ctypes.c_void_p(self.stream.cuda_stream)
        g = torch.Generator().manual_seed(seed)
        # All weights, then all biases, in flat FP32 buffers (master values,
        # gradients, Adam moments) and one BF16 copy: the optimizer step, the
        # gradient reset and the BF16 copy are one launch each.
        self.n_w = sum(co * ci * k * k for co, ci, k in self.shapes.values())
        n_all = self.n_w + sum(co for co, _, _ in self.shapes.values())
        self.flat = {key: torch.zeros(n_all, device=self.dev) for key in ("w", "g", "m", "v")}
        self.flat["wb"] = torch.zeros(n_all, dtype=torch.bfloat16, device=self.dev)
        self.params = {}
        self._offsets = {}
        wo, bo = 0, self.n_w
        for name, (co, ci, k) in self.shapes.items():
            std = (2.0 / (ci * k * k)) ** 0.5
            wm = (torch.randn((co, ci, k, k), generator=g, dtype=torch.float64) * std).float().to(self.dev)
            self._offsets[name] = (wo, bo)
            self.params[name] = self._param(name, wm, torch.zeros(co, device=self.dev))
            wo += co * ci * k * k
            bo += co
        self._pack_jobs()
        self.step_count = 0
        self.norm = dict(rho_mean=1.5, rho_std=1.0, u_scale=1e-3)
        self._wc_cache = {}
        self.train_graph = None
        self._alloc(batch)

    def _param(self, name, wm, bm):
        t = self.torch
        co, ci, k = self.shapes[name]
        wo, bo = self._offsets[name]
        nw = co * ci * k * k
        fw = lambda key: self.flat[key][wo:wo + nw].view(co, ci, k, k)  # noqa: E731
        fb = lambda key: self.flat[key][bo:bo + co]  # noqa: E731
        p = dict(w=fw("w"), b=fb("w"), wb=fw("wb"), gw=fw("g"), gb=fb("g"), mw=fw("m"), vw=fw("v"), mb=fb("m"),
                 vb=fb("v"))
        p["w"].copy_(wm)
        p["b"].copy_(bm)
        if k == 3:
            p["wt"] = t.empty(int(self.lib.unet_conv_pack_elems(co, ci, 0)), dtype=t.bfloat16, device=self.dev)
            if ci % 32 == 0:  # the input gradient of the first layer is not needed
                p["wtT"] = t.empty(int(self.lib.unet_conv_pack_elems(co, ci, 1)), dtype=t.bfloat16, device=self.dev)
        self._refresh(name, p)
        return p

    def _refresh(self, name, p):
        """BF16 compute copy and packed tensor-core operands from the FP32 master weights."""
        co, ci, k = self.shapes[name]
        _call(self.lib.unet_f32_to_bf16, ctypes.c_void_p(p["w"].data_ptr()), ctypes.c_void_p(p["wb"].data_ptr()),
              p["w"].numel(), self.s)
        if k == 3:
            _call(self.lib.unet_conv_pack, ctypes.c_void_p(p["w"].data_ptr()), co, ci, 0,
                  ctypes.c_void_p(p["wt"].data_ptr()), self.s)
            if "wtT" in p:
                _call(self.lib.unet_conv_pack, ctypes.c_void_p(p["w"].data_ptr()), co, ci, 1,
                      ctypes.c_void_p(p["wtT"].data_ptr()), self.s)

    def _pack_jobs(self):
        """Device table of every layer's packings (unet_conv_pack_many)."""
        jobs, most = [], 1
        for name, p in self.params.items():
            co, ci, k = self.shapes[name]
            for tr, key in ((0, "wt"), (1, "wtT")):
                if key in p:
                    jobs.append([p["w"].data_ptr(), co, ci, tr, p[key].data_ptr()])
                    most = max(most, int(self.lib.unet_conv_pack_elems(co, ci, tr)))
        self.pack_table = self.torch.tensor(jobs, dtype=self.torch.int64, device=self.dev)
        self.pack_most = most

    def _refresh_packs(self):
        """Packed tensor-core operands of every layer from the FP32 master
        weights (one launch; the optimizer writes the BF16 copies itself)."""
        _call(self.lib.unet_conv_pack_many, ctypes.c_void_p(self.pack_table.data_ptr()),
              int(self.pack_table.shape[0]), self.pack_most, self.s)

    def set_weights(self, weights: dict):
        """Load FP32 weights/biases {name: (w, b)} (e.g. to match a reference)."""
        for name, (w, b) in weights.items():
            p = self.params[name]
            p["w"].copy_(self.torch.as_tensor(w, dtype=self.torch.float32))
            p["b"].copy_(self.torch.as_tensor(b, dtype=self.torch.float32))
            self._refresh(name, p)

    def weights(self) -> dict:
        return {k: (p["w"].detach().cpu().numpy(), p["b"].detach().cpu().numpy()) for k, p in self.params.items()}

    def _alloc(self, B):
        t = self.torch
        H, W = self.H, self.W
        bf = dict(dtype=t.bfloat16, device=self.dev)
        hw = [(H >> l, W >> l) for l in range(4)]
        self.x0 = t.zeros((B, H, W, IN_PAD), **bf)
        self.A = [t.zeros((B, *hw[l], C[l]), **bf) for l in range(4)]
        self.B3 = t.zeros((B, *hw[3], C[3]), **bf)
        self.cat = [t.zeros((B, *hw[l], C[l + 1] + C[l]), **bf) for l in range(3)]
        self.P = [t.zeros((B, *hw[l + 1], C[l]), **bf) for l in range(3)]
        self.DA = [t.zeros((B, *hw[l], C[l]), **bf) for l in range(3)]
        self.DB = [t.zeros((B, *hw[l], C[l]), **bf) for l in range(3)]
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
        co, ci, _ = self.shapes[name]
        _call(self.lib.unet_conv3x3, x.ptr, x.ct, ci, ctypes.c_void_p(p["wt"].data_ptr()),
              ctypes.c_void_p(p["b"].data_ptr()), y.ptr, y.ct, co, self.batch, h, w, 1 if relu else 0, self.s)

    def _conv_bwd(self, name, x: View, y: View, gy: View, gx: View | None, h, w):
        """Through relu(conv(x)): gy *= (y > 0); accumulate weight/bias grads;
        gx = conv^T(gy) if gx is given."""
        p = self.params[name]
        co, ci, _ = self.shapes[name]
        lib, n = self.lib, self.batch
        _call(lib.unet_relu_bwd, y.ptr, y.ct, gy.ptr, gy.ct, co, n * h * w, ctypes.c_void_p(p["gb"].data_ptr()),
              self.s)
        _call(lib.unet_conv3x3_bwd_weight, x.ptr, x.ct, ci, gy.ptr, gy.ct, co,
              ctypes.c_void_p(p["gw"].data_ptr()), None, n, h, w, self.s)
        if gx is not None:
            _call(lib.unet_conv3x3, gy.ptr, gy.ct, co, ctypes.c_void_p(p["wtT"].data_ptr()), None, gx.ptr, gx.ct,
                  ci, n, h, w, 0, self.s)

    def forward(self, x_planes):
        """x_planes: float tensor [B, in_ch, H, W] on the device -> self.out (FP32, [B, 3, H, W])."""
        lib, n, s = self.lib, self.batch, self.s
        H, W = self.H, self.W
        xs = x_planes.contiguous().float()
        _call(lib.unet_input_nhwc, ctypes.c_void_p(xs.data_ptr()), xs.shape[1], H * W, n,
              ctypes.c_void_p(self.x0.data_ptr()), IN_PAD, s)
        h = View(self.x0, 0, self.in_ch)
        for l in range(4):
            hh, ww = H >> l, W >> l
            a = View(self.A[l], 0, C[l])
            self._conv(f"e{l}a", h, a, hh, ww)
            if l < 3:
                skip = View(self.cat[l], C[l + 1], C[l])
                self._conv(f"e{l}b", a, skip, hh, ww)
                _call(lib.unet_pool2_fwd, skip.ptr, skip.ct, ctypes.c_void_p(self.P[l].data_ptr()), C[l], C[l], n,
                      hh, ww, s)
                h = View(self.P[l], 0, C[l])
            else:
                self._conv("e3b", a, View(self.B3, 0, C[3]), hh, ww)
        lower = View(self.B3, 0, C[3])
        for l in (2, 1, 0):
            hh, ww = H >> l, W >> l
            up = View(self.cat[l], 0, C[l + 1])
            _call(lib.unet_up2_fwd, lower.ptr, lower.ct, up.ptr, up.ct, C[l + 1], n, hh // 2, ww // 2, s)
            self._conv(f"d{l}a", View(self.cat[l], 0, C[l + 1] + C[l]), View(self.DA[l], 0, C[l]), hh, ww)
            self._conv(f"d{l}b", View(self.DA[l], 0, C[l]), View(self.DB[l], 0, C[l]), hh, ww)
            lower = View(self.DB[l], 0, C[l])
        hp = self.params["head"]
        _call(lib.unet_head_fwd, lower.ptr, lower.ct, C[0], ctypes.c_void_p(hp["wb"].data_ptr()),
              ctypes.c_void_p(hp["b"].data_ptr()), ctypes.c_void_p(self.out.data_ptr()), OUT_CH, n, H * W, s)
        return self.out

    def loss_backward(self, target, wc, sync=True):
        """MSE against target [B, 3, H, W] (FP32) with channel weights wc;
        fills every parameter gradient (zeroed first); returns the loss
        (a float, or with sync=False the FP64 device scalar)."""
        t, lib, n, s = self.torch, self.lib, self.batch, self.s
        H, W = self.H, self.W
        self.flat["g"].zero_()
        self.loss_acc.zero_()
        tg = target.contiguous().float()
        wct = self._wc_dev(wc)
        _call(lib.unet_mse, ctypes.c_void_p(self.out.data_ptr()), ctypes.c_void_p(tg.data_ptr()),
              ctypes.c_void_p(wct.data_ptr()), OUT_CH, H * W, self.out.numel(),
              ctypes.c_void_p(self.gout.data_ptr()), ctypes.c_void_p(self.loss_acc.data_ptr()), s)
        hp = self.params["head"]
        db0, gdb0 = View(self.DB[0], 0, C[0]), View(self.gDB[0], 0, C[0])
        _call(lib.unet_head_bwd, db0.ptr, db0.ct, C[0], ctypes.c_void_p(hp["wb"].data_ptr()),
              ctypes.c_void_p(self.gout.data_ptr()), OUT_CH, n, H * W, gdb0.ptr, gdb0.ct,
              ctypes.c_void_p(hp["gw"].data_ptr()), ctypes.c_void_p(hp["gb"].data_ptr()), s)
        gup = None
        for l in (0, 1, 2):
            hh, ww = H >> l, W >> l
            if gup is not None:
                # gradient of level l's decoder output arrives through the upsampling
                g = View(self.gDB[l], 0, C[l])
                _call(lib.unet_up2_bwd, gup.ptr, gup.ct, g.ptr, g.ct, C[l], n, hh, ww, s)
            self._conv_bwd(f"d{l}b", View(self.DA[l], 0, C[l]), View(self.DB[l], 0, C[l]),
                           View(self.gDB[l], 0, C[l]), View(self.gDA[l], 0, C[l]), hh, ww)
            self._conv_bwd(f"d{l}a", View(self.cat[l], 0, C[l + 1] + C[l]), View(self.DA[l], 0, C[l]),
                           View(self.gDA[l], 0, C[l]), View(self.gcat[l], 0, C[l + 1] + C[l]), hh, ww)
            gup = View(self.gcat[l], 0, C[l + 1])  # towards the level below (coarser)
        # bottleneck: gradient of B3 through the level-2 upsampling
        hh, ww = H >> 3, W >> 3
        g3 = View(self.gB3, 0, C[3])
        _call(lib.unet_up2_bwd, gup.ptr, gup.ct, g3.ptr, g3.ct, C[3], n, hh, ww, s)
        self._conv_bwd("e3b", View(self.A[3], 0, C[3]), View(self.B3, 0, C[3]), g3, View(self.gA[3], 0, C[3]), hh, ww)
        self._conv_bwd("e3a", View(self.P[2], 0, C[2]), View(self.A[3], 0, C[3]), View(self.gA[3], 0, C[3]),
                       View(self.gP[2], 0, C[2]), hh, ww)
        for l in (2, 1, 0):
            hh, ww = H >> l, W >> l
            gskip = View(self.gcat[l], C[l + 1], C[l])
            gp = View(self.gP[l], 0, C[l])
            _call(lib.unet_pool2_bwd, gp.ptr, gp.ct, gskip.ptr, gskip.ct, C[l], n, hh, ww, 1, s)
            self._conv_bwd(f"e{l}b", View(self.A[l], 0, C[l]), View(self.cat[l], C[l + 1], C[l]), gskip,
                           View(self.gA[l], 0, C[l]), hh, ww)
            below = View(self.x0, 0, self.in_ch) if l == 0 else View(self.P[l - 1], 0, C[l - 1])
            self._conv_bwd(f"e{l}a", below, View(self.A[l], 0, C[l]), View(self.gA[l], 0, C[l]),
                           None if l == 0 else View(self.gP[l - 1], 0, C[l - 1]), hh, ww)
        return float(self.loss_acc.item()) if sync else self.loss_acc.clone()

    def _wc_dev(self, wc):
        """Channel weights of the loss as a device tensor (made once per value,
        so that a captured training step copies nothing from the host)."""
        key = tuple(float(v) for v in wc)
        d = self._wc_cache.get(key)
        if d is None:
            d = self.torch.tensor(key, dtype=self.torch.float32, device=self.dev)
            self._wc_cache[key] = d
        return d

    def adam(self, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=0.0, hyper=None):
        """One Adam step. hyper (device address of lr, 1 - beta1^t, 1 - beta2^t,
        written by unet_adam_hyper) replaces lr and the host step count."""
        if hyper is None:
            self.step_count += 1
        f = self.flat
        n_all = f["w"].numel()
        # weight decay on the weights only: one launch over everything without it
        ranges = [(0, n_all, weight_decay)] if weight_decay == 0.0 else \
            [(0, self.n_w, weight_decay), (self.n_w, n_all, 0.0)]
        for a, b, wd in ranges:
            args = tuple(ctypes.c_void_p(f[key].data_ptr() + a * f[key].element_size())
                         for key in ("w", "wb", "g", "m", "v")) + (b - a,)
            if hyper is None:
                _call(self.lib.unet_adam, *args, lr, beta1, beta2, eps, self.step_count, wd, self.s)
            else:
                _call(self.lib.unet_adam_dev, *args, ctypes.c_void_p(hyper), beta1, beta2, eps, wd, self.s)
        self._refresh_packs()

    def make_train_graph(self, wc, lr_schedule, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=0.0):
        """Capture one training step (forward, loss and backward, Adam) as a
        CUDA graph reading its input planes from self.g_in and its targets
        from self.g_tg; replay k uses learning rate lr_schedule[k] (the last
        entry beyond the end) and continues the Adam step count on the
        device (self.adam_state, see unet_adam_hyper)."""
        import numpy as np
        t = self.torch
        self.g_in = t.zeros((self.B, self.in_ch, self.H, self.W), device=self.dev)
        self.g_tg = t.zeros((self.B, OUT_CH, self.H, self.W), device=self.dev)
        p1, p2 = np.float32(1.0), np.float32(1.0)
        for _ in range(self.step_count):  # the running products of the host path, in FP32
            p1, p2 = np.float32(p1 * np.float32(beta1)), np.float32(p2 * np.float32(beta2))
        self.adam_state = t.tensor([float(self.step_count), float(p1), float(p2), 0.0, 0.0, 0.0],
                                   dtype=t.float32, device=self.dev)
        self.lr_sched = t.tensor([float(v) for v in lr_schedule], dtype=t.float32, device=self.dev)
        self._wc_dev(wc)
        side = t.cuda.Stream()
        side.wait_stream(self.stream)
        old = (self.stream, self.s)
        self.stream, self.s = side, ctypes.c_void_p(side.cuda_stream)
        try:
            with t.cuda.stream(side):
                # one pass without the optimizer step before capture (lazy set-up)
                self.forward(self.g_in)
                self.loss_backward(self.g_tg, wc, sync=False)
            side.synchronize()
            g = t.cuda.CUDAGraph()
            with t.cuda.graph(g, stream=side):
                _call(self.lib.unet_adam_hyper, ctypes.c_void_p(self.adam_state.data_ptr()),
                      ctypes.c_void_p(self.lr_sched.data_ptr()), int(self.lr_sched.numel()), beta1, beta2, self.s)
                self.forward(self.g_in)
                self.loss_backward(self.g_tg, wc, sync=False)
                self.adam(beta1=beta1, beta2=beta2, eps=eps, weight_decay=weight_decay,
                          hyper=self.adam_state.data_ptr() + 3 * 4)
        finally:
            self.stream, self.s = old
        self.stream.wait_stream(side)
        self.train_graph = g
        return g

    def replay_train_step(self, planes, targets):
        """One captured training step on the given batch (copied into the
        graph's input and target buffers on the network's stream); the loss
        lands in self.loss_acc."""
        t = self.torch
        with t.cuda.stream(self.stream):
            self.g_in.copy_(planes)
            self.g_tg.copy_(targets)
            self.train_graph.replay()
        self.step_count += 1

    def check_tensor_cores(self):
        """Raise if a tensor-core kernel's bounded wait timed out (flag cleared)."""
        if self.lib.unet_tc_error(self.s, 1) != 0:
            raise RuntimeError("a tensor-core kernel timed out waiting for its MMAs")

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

    def predict_raw(self, planes):
        """Normalised network output [N, 3, H, W] (FP32, device) for input
        planes [N, 3, H, W], N any size (run in batches of the network's batch)."""
        t = self.torch
        n = planes.shape[0]
        out = t.empty((n, OUT_CH, self.H, self.W), dtype=t.float32, device=self.dev)
        for i in range(0, n, self.batch):
            chunk = planes[i:i + self.batch]
            k = chunk.shape[0]
            if k < self.batch:
                chunk = t.cat([chunk, chunk[-1:].expand(self.batch - k, -1, -1, -1)])
            out[i:i + k] = self.forward(chunk)[:k]
        return out

    def predict(self, planes):
        """Decoded (rho, u_x, u_y) device tensors [N, H, W] for input planes."""
        return self.decode(self.predict_raw(planes))

    def warm_fields(self, planes, masks, mass, rho_range):
        """Initial (rho, u_x, u_y) of N domains as one FP64 device tensor
        [N, 3, H, W] (each [3, H, W] slice in the LBM_RHO_U_PHYS layout): the
        decoded prediction with rho clamped to rho_range on fluid nodes, 0 on
        solids, and each domain's rho scaled to sum to mass[i] (the method
        conserves mass, and its steady state depends on it). masks: [N, H, W]
        (1 = solid); mass: N values."""
        t = self.torch
        raw = self.predict_raw(planes)
        n = raw.shape[0]
        m = t.as_tensor(np.asarray(masks), dtype=t.uint8, device=self.dev).contiguous()
        ms = t.as_tensor(np.asarray(mass, dtype=np.float64), device=self.dev)
        out = t.empty((n, OUT_CH, self.H, self.W), dtype=t.float64, device=self.dev)
        sums = t.empty(n, dtype=t.float64, device=self.dev)
        nm = self.norm
        _call(self.lib.unet_warm_fields, ctypes.c_void_p(raw.data_ptr()), n, self.H * self.W,
              ctypes.c_void_p(m.data_ptr()), ctypes.c_void_p(ms.data_ptr()), nm["rho_mean"], nm["rho_std"],
              nm["u_scale"], float(rho_range[0]), float(rho_range[1]), ctypes.c_void_p(out.data_ptr()),
              ctypes.c_void_p(sums.data_ptr()), self.s)
        return out


# ---------------------------------------------------------------- warm start
def channel_planes(net, ws):
    """Input planes of the surrogate for channel workloads (mask, level, fill)."""
    return net.planes(np.stack([w.mask for w in ws]), [w.meta["level"] for w in ws],
                      [w.meta["fill"] for w in ws])


def flat_walls(mask) -> bool:
    """True if the walls run parallel to x (every column has the same solid
    rows): the steady state of such a channel does not depend on the start.
    Rough walls hold vapor pockets in their grooves, and where the pockets
    settle depends on the path to the steady state, so a warm start could
    converge to another steady flux than the cold start."""
    m = np.asarray(mask)
    return bool(np.all(m == m[:, :1]))


def steady_states(ws, stream=None, rel_tol=1e-7, check_every=1000, max_steps=60000, chunk=1024, storage=None):
    """Run every workload from its cold start to steady flux (batched) and
    return a dict of device tensors: fields [N, 3, ny, nx] FP32 (rho, u_x,
    u_y), steps [N] (-1: not steady within max_steps, -2: non-finite) and
    flux Q [N] (FP64)."""
    import torch
    from . import lbm as L
    storage = L.LBM_FP32_DEV if storage is None else storage
    fields, steps, flux = [], [], []
    for i in range(0, len(ws), chunk):
        part = ws[i:i + chunk]
        b = L.Batch([dict(nx=w.nx, ny=w.ny, storage=storage, **w.params) for w in part], stream=stream)
        try:
            for w, d in zip(part, b.domains):
                d.set_geometry(w.mask)
                d.set_rho_u(w.rho)
            st, obs, _ = b.run_to_steady(rel_tol, check_every, max_steps)
            for d in b.domains:
                fields.append(d.fields_device().float())
        finally:
            b.close()
        steps += st
        flux += [o["flux_Q"] for o in obs]
    return dict(fields=torch.stack(fields), steps=torch.tensor(steps), flux=torch.tensor(flux, dtype=torch.float64))


def fit_normalisation(net, fields, mask):
    """Density mean/std over fluid nodes and the velocity scale (largest |u_x|)."""
    fl = mask == 0
    rho = fields[:, 0][fl]
    net.norm = dict(rho_mean=float(rho.mean()), rho_std=float(rho.std()),
                    u_scale=float(fields[:, 1][fl].abs().max()))
    return net.norm


def train(net, planes, targets, epochs=20, lr=2e-3, wc=(1.0, 1.0, 0.25), seed=0, lr_final=1e-4, graph=True):
    """Adam over shuffled mini-batches (the network's batch size) with a
    cosine learning-rate decay from lr to lr_final; returns the mean loss of
    every epoch. graph: replay one captured CUDA graph per step (the same
    kernels and values as the step-by-step launches, without the host cost
    of about 200 launches per step)."""
    import math
    t = net.torch
    g = t.Generator().manual_seed(seed)
    n = planes.shape[0]
    per_epoch = n // net.batch
    total = epochs * per_epoch
    rates = [lr_final + 0.5 * (lr - lr_final) * (1 + math.cos(math.pi * k / max(1, total - 1)))
             for k in range(total)]
    if graph:
        net.make_train_graph(wc, rates)
    history = []
    k = 0
    for _ in range(epochs):
        perm = t.randperm(n, generator=g).to(planes.device)
        acc = t.zeros(1, dtype=t.float64, device=planes.device)
        for j in range(per_epoch):
            idx = perm[j * net.batch:(j + 1) * net.batch]
            if graph:
                net.replay_train_step(planes[idx], targets[idx])
                with t.cuda.stream(net.stream):
                    acc += net.loss_acc
            else:
                net.forward(planes[idx])
                acc += net.loss_backward(targets[idx], wc, sync=False)
                net.adam(lr=rates[k])
            k += 1
        history.append(float(acc.item()) / per_epoch)
    return history


def fit(ws, epochs=40, lr=2e-3, batch=16, seed=0, stream=None, wc=(1.0, 1.0, 0.25), **steady_kw):
    """Generate the steady states of ``ws`` with the method itself, then
    train a surrogate on them with the hand-written kernels. Returns the
    network (norm set) and a dict of timings and the loss history."""
    import time
    import torch
    info = {}
    t0 = time.perf_counter()
    data = steady_states(ws, stream=stream, **steady_kw)
    torch.cuda.synchronize()
    info["generate_s"] = time.perf_counter() - t0
    keep = data["steps"] > 0
    info["samples"] = int(keep.sum())
    net = UNet(batch=batch, height=ws[0].ny, width=ws[0].nx, seed=seed, stream=stream)
    fields = data["fields"][keep.to(data["fields"].device)]
    masks = torch.as_tensor(np.stack([w.mask for w, k in zip(ws, keep.tolist()) if k]), device=fields.device)
    fit_normalisation(net, fields, masks)
    planes = channel_planes(net, [w for w, k in zip(ws, keep.tolist()) if k])
    targets = fields.clone()
    targets[:, 0] = (targets[:, 0] - net.norm["rho_mean"]) / net.norm["rho_std"]
    targets[:, 1:] /= net.norm["u_scale"]
    targets = torch.where(masks[:, None] == 0, targets, 0.0)
    t0 = time.perf_counter()
    info["loss"] = train(net, planes, targets, epochs=epochs, lr=lr, wc=wc, seed=seed)
    torch.cuda.synchronize()
    info["train_s"] = time.perf_counter() - t0
    # fit on (up to 64 of) the training states, relative L2 over fluid nodes
    k = min(64, planes.shape[0])
    rho, ux, _ = net.predict(planes[:k])
    fl = masks[:k] == 0
    info["train_rel_l2"] = {
        "rho": float(torch.linalg.norm((rho - fields[:k, 0])[fl]) / torch.linalg.norm(fields[:k, 0][fl])),
        "u_x": float(torch.linalg.norm((ux - fields[:k, 1])[fl]) / torch.linalg.norm(fields[:k, 1][fl]))}
    return net, info


def cold_mass(w) -> float:
    """Mass of a workload's cold start (sum of rho over fluid nodes)."""
    return float(np.sum(np.where(w.mask == 0, w.rho, 0.0)))


def batch_run_to_steady(ws, net=None, stream=None, rel_tol=1e-7, check_every=1000, max_steps=60000,
                        storage=None, policy=flat_walls, probe_checks=2, fallback_tol=0.05):
    """All workloads in one batch, run to steady flux; with a surrogate
    ``net``, the domains that ``policy`` accepts start from its prediction.

    A warm-started domain is set through LBM_RHO_U_PHYS (the predicted u is
    the physical velocity). After ``probe_checks`` convergence intervals, a
    warm-started domain restarts from its cold start if it went non-finite,
    or if its flux residual |dQ|/|Q| per interval is still above
    ``fallback_tol`` and did not drop over the probe (a cold start's
    residual after two intervals is of order 1, a useful warm start's
    1e-2 or less); the run then goes on
    to convergence as lbm_batch_run_to_steady defines it. Returns (steps [N]
    counted from the first step, including any probe before a restart, obs
    list, info) with info = {warm, restarted: [N] flags, probe_residuals:
    [N] lists}."""
    from . import lbm as L
    storage = L.LBM_FP32_DEV if storage is None else storage
    from . import workloads as wl
    warm = [net is not None and bool(policy(w.mask)) for w in ws]
    fields = None
    if any(warm):
        sel = [w for w, f in zip(ws, warm) if f]
        fields = net.warm_fields(channel_planes(net, sel), np.stack([w.mask for w in sel]),
                                 [cold_mass(w) for w in sel], (0.5 * wl.RHO_V, 1.1 * wl.RHO_L))
    b = L.Batch([dict(nx=w.nx, ny=w.ny, storage=storage, **w.params) for w in ws], stream=stream)
    info = dict(warm=warm, restarted=[False] * len(ws), probe_residuals=[[] for _ in ws])
    try:
        k = 0
        for w, d, f in zip(ws, b.domains, warm):
            d.set_geometry(w.mask)
            if f:
                d.set_rho_u_field(fields[k], physical=True)
                k += 1
            else:
                d.set_rho_u(w.rho)
        if any(warm) and probe_checks > 0:
            q = [[o["flux_Q"] for o in b.observables(check_finite=False)]]
            for _ in range(probe_checks):
                b.step(check_every)
                q.append([o["flux_Q"] if o["nonfinite"] == 0 else float("nan")
                          for o in b.observables(check_finite=False)])
            for i, (w, d) in enumerate(zip(ws, b.domains)):
                if not warm[i]:
                    continue
                res = [abs(q[j + 1][i] - q[j][i]) / max(abs(q[j + 1][i]), 1e-300) for j in range(probe_checks)]
                info["probe_residuals"][i] = res
                stuck = res[-1] > fallback_tol and res[-1] >= res[0]
                if not all(np.isfinite(res)) or stuck:
                    d.set_rho_u(w.rho)
                    info["restarted"][i] = True
        steps, obs, _ = b.run_to_steady(rel_tol, check_every, max_steps)
    finally:
        b.close()
    return steps, obs, info


def _time_training_step(argv=None):
    """Time forward + backward + Adam of one network on random planes (CUDA
    events around `steps` steps after `warmup` steps); prints ms per step."""
    import argparse
    import torch
    ap = argparse.ArgumentParser(description=_time_training_step.__doc__)
    ap.add_argument("--batch", type=int, default=16)
    ap.add_argument("--height", type=int, default=64)
    ap.add_argument("--width", type=int, default=256)
    ap.add_argument("--warmup", type=int, default=4)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--eager", action="store_true", help="launch step by step instead of one CUDA graph per step")
    a = ap.parse_args(argv)
    net = UNet(batch=a.batch, height=a.height, width=a.width, seed=0)
    g = torch.Generator().manual_seed(0)
    planes = torch.rand((a.batch, IN_CH, a.height, a.width), generator=g).cuda()
    target = torch.randn((a.batch, OUT_CH, a.height, a.width), generator=g).cuda()

    if a.eager:
        def step():
            net.forward(planes)
            net.loss_backward(target, [1.0, 1.0, 1.0], sync=False)
            net.adam(1e-3)
    else:
        net.make_train_graph([1.0, 1.0, 1.0], [1e-3])

        def step():
            net.replay_train_step(planes, target)

    for _ in range(a.warmup):
        step()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(a.steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    net.check_tensor_cores()
    print(f"U-Net training step, batch {a.batch} of {a.height}x{a.width} "
          f"({'step-by-step launches' if a.eager else 'one CUDA graph per step'}): "
          f"{e0.elapsed_time(e1) / max(1, a.steps):.3f} ms")


if __name__ == "__main__":
    _time_training_step()
