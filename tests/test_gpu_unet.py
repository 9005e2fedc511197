"""U-Net kernels and network against the CPU reference (oracle/unet_oracle).

Activations are BF16 channels-last; the 3x3 convolutions and their
gradients run on the tensor cores. The reference gets the same BF16-rounded
weights and inputs in FP64, so the remaining differences are accumulation
order and the BF16 rounding of outputs and of intermediate activations and
gradients. Bounds: single kernels 1e-2 relative (L2) of the output; the whole
network's output 3e-2 and every layer's weight gradient 8e-2 relative (L2)
after the 16 layers of BF16 round trips. Views are exercised as channel
ranges of wider buffers.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0708_4182_gb300 import surrogate
    lib = surrogate.load_unet()
    yield torch, surrogate, lib
    assert lib.unet_tc_error(ctypes.c_void_p(torch.cuda.current_stream().cuda_stream), 1) == 0


def rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def ref_conv(x, w, b=None):
    import torch.nn.functional as F
    xp = F.pad(F.pad(x, (1, 1, 0, 0), mode="circular"), (0, 0, 1, 1))
    return F.conv2d(xp, w, b)


def vp(t, c0=0):
    return ctypes.c_void_p(t.data_ptr() + c0 * t.element_size())


def nhwc_buffer(t, x_nchw, extra, off):
    """BF16 NHWC buffer with `extra` more channels than x, x stored at channel `off`."""
    n, c, h, w = x_nchw.shape
    buf = t.zeros((n, h, w, c + extra), dtype=t.bfloat16, device="cuda")
    buf[..., off:off + c] = x_nchw.permute(0, 2, 3, 1).to(t.bfloat16).cuda()
    return buf


@pytest.mark.parametrize("ci,co,h,w", [(3, 32, 64, 256), (96, 32, 32, 64), (32, 64, 32, 32), (256, 128, 8, 32),
                                       (384, 128, 8, 32), (64, 96, 8, 64),
                                       # 1 and 3 chunks of 16 input channels (one chunk per ring slot)
                                       (16, 32, 8, 64), (48, 64, 8, 32),
                                       # images >= 128 wide: the one-row halo kernel
                                       (64, 128, 8, 128), (32, 64, 4, 256), (96, 32, 8, 128), (192, 64, 4, 128)])
def test_conv3x3_forward_backward(env, ci, co, h, w):
    t, surrogate, lib = env
    g = t.Generator().manual_seed(ci + co)
    n = 2
    s = ctypes.c_void_p(t.cuda.current_stream().cuda_stream)
    x = t.randn((n, ci, h, w), generator=g).to(t.bfloat16).double()
    wt = (t.randn((co, ci, 3, 3), generator=g) * (2.0 / (9 * ci)) ** 0.5).to(t.bfloat16)
    b = t.randn(co, generator=g) * 0.1
    dy = t.randn((n, co, h, w), generator=g).to(t.bfloat16).double()
    # input view: channels [8, 8 + ci) of a wider buffer (ci = 3: 16 readable zero-padded channels)
    pad_in = 16 - ci if ci < 16 else 0
    xoff = 0 if ci < 16 else 8
    xb = nhwc_buffer(t, x, pad_in + (0 if ci < 16 else 16), xoff)
    wm = wt.float().cuda().contiguous()
    packed = t.empty(int(lib.unet_conv_pack_elems(co, ci, 0)), dtype=t.bfloat16, device="cuda")
    assert lib.unet_conv_pack(vp(wm), co, ci, 0, vp(packed), s) == 0
    yb = t.zeros((n, h, w, co + 32), dtype=t.bfloat16, device="cuda")  # output at channel 16
    bias = b.float().cuda()
    assert lib.unet_conv3x3(vp(xb, xoff), xb.shape[-1], ci, vp(packed), vp(bias), vp(yb, 16), yb.shape[-1], co,
                            n, h, w, 1, s) == 0
    ref = t.relu(ref_conv(x, wt.double(), b.double()))
    got = yb[..., 16:16 + co].permute(0, 3, 1, 2).float().cpu()
    assert rel(got, ref) < 1e-2
    assert t.all(yb[..., :16] == 0) and t.all(yb[..., 16 + co:] == 0)  # nothing outside the view
    # gradient w.r.t. the input (no activation): transposed packing, needs ci % 32 == 0
    xr = x.clone().requires_grad_(True)
    wr = wt.double().requires_grad_(True)
    br = t.zeros(co, dtype=t.float64, requires_grad=True)
    (ref_conv(xr, wr, br) * dy).sum().backward()
    dyb = nhwc_buffer(t, dy, 8, 8)
    if ci % 32 == 0:
        packT = t.empty(int(lib.unet_conv_pack_elems(co, ci, 1)), dtype=t.bfloat16, device="cuda")
        assert lib.unet_conv_pack(vp(wm), co, ci, 1, vp(packT), s) == 0
        dxb = t.zeros((n, h, w, ci), dtype=t.bfloat16, device="cuda")
        assert lib.unet_conv3x3(vp(dyb, 8), dyb.shape[-1], co, vp(packT), None, vp(dxb), ci, ci, n, h, w, 0, s) == 0
        assert rel(dxb.permute(0, 3, 1, 2).float().cpu(), xr.grad) < 1e-2
    # gradients w.r.t. weights and bias (accumulated: start from a known value)
    dw = t.full((co, ci, 3, 3), 0.5, device="cuda")
    db = t.full((co,), 0.25, device="cuda")
    assert lib.unet_conv3x3_bwd_weight(vp(xb, xoff), xb.shape[-1], ci, vp(dyb, 8), dyb.shape[-1], co, vp(dw), vp(db),
                                       n, h, w, s) == 0
    assert rel(dw.cpu() - 0.5, wr.grad) < 1e-2
    assert rel(db.cpu() - 0.25, br.grad) < 1e-2


def test_pool_upsample_head_relu(env):
    t, surrogate, lib = env
    import torch.nn.functional as F
    g = t.Generator().manual_seed(7)
    n, c, h, w = 2, 32, 16, 64
    s = ctypes.c_void_p(t.cuda.current_stream().cuda_stream)
    x = t.randn((n, c, h, w), generator=g).to(t.bfloat16).double()
    xb = nhwc_buffer(t, x, 16, 8)
    p = t.zeros((n, h // 2, w // 2, c), dtype=t.bfloat16, device="cuda")
    assert lib.unet_pool2_fwd(vp(xb, 8), xb.shape[-1], vp(p), c, c, n, h, w, s) == 0
    assert rel(p.permute(0, 3, 1, 2).float().cpu(), F.avg_pool2d(x, 2)) < 1e-2
    u = t.zeros((n, h, w, c + 8), dtype=t.bfloat16, device="cuda")
    assert lib.unet_up2_fwd(vp(p), c, vp(u, 8), u.shape[-1], c, n, h // 2, w // 2, s) == 0
    want = F.interpolate(p.permute(0, 3, 1, 2).float().cpu(), scale_factor=2, mode="nearest")
    assert t.equal(u[..., 8:].permute(0, 3, 1, 2).float().cpu(), want)
    # adjoints: <pool(x), y> = <x, pool^T(y)>, <up(a), b> = <a, up^T(b)>
    yb = t.randn((n, c, h // 2, w // 2), generator=g).to(t.bfloat16).double()
    ybn = nhwc_buffer(t, yb, 0, 0)
    dx = t.zeros((n, h, w, c), dtype=t.bfloat16, device="cuda")
    assert lib.unet_pool2_bwd(vp(ybn), c, vp(dx), c, c, n, h, w, 0, s) == 0
    lhs = (F.avg_pool2d(x, 2) * yb).sum().item()
    assert abs(lhs - (x * dx.permute(0, 3, 1, 2).double().cpu()).sum().item()) < 2e-2 * abs(lhs) + 1e-3
    # accumulating form: adds the same adjoint onto what dx holds
    before = dx.clone()
    assert lib.unet_pool2_bwd(vp(ybn), c, vp(dx), c, c, n, h, w, 1, s) == 0
    assert rel((dx.float() - before.float()).cpu(), before.float().cpu()) < 1e-2
    bb = t.randn((n, c, h, w), generator=g).to(t.bfloat16).double()
    bbn = nhwc_buffer(t, bb, 0, 0)
    da = t.zeros((n, h // 2, w // 2, c), dtype=t.bfloat16, device="cuda")
    assert lib.unet_up2_bwd(vp(bbn), c, vp(da), c, c, n, h // 2, w // 2, s) == 0
    lhs = (F.interpolate(yb, scale_factor=2, mode="nearest") * bb).sum().item()
    assert abs(lhs - (yb * da.permute(0, 3, 1, 2).double().cpu()).sum().item()) < 2e-2 * abs(lhs) + 1e-3
    # 1x1 head (NHWC in, FP32 NCHW out)
    wh = t.randn((3, c, 1, 1), generator=g).to(t.bfloat16)
    bh = t.randn(3, generator=g).float().cuda()
    yh = t.empty((n, 3, h, w), device="cuda")
    whc = wh.reshape(3, c).contiguous().cuda()
    assert lib.unet_head_fwd(vp(xb, 8), xb.shape[-1], c, vp(whc), vp(bh), vp(yh), 3, n, h * w, s) == 0
    assert rel(yh.cpu(), F.conv2d(x, wh.double(), bh.double().cpu())) < 1e-3
    # ReLU backward on views
    gyb = nhwc_buffer(t, bb, 8, 0)
    dbr = t.full((c,), 0.5, device="cuda")
    assert lib.unet_relu_bwd(vp(xb, 8), xb.shape[-1], vp(gyb), gyb.shape[-1], c, n * h * w, vp(dbr), s) == 0
    want = t.where(x > 0, bb, t.zeros_like(bb))
    assert t.equal(gyb[..., :c].permute(0, 3, 1, 2).double().cpu(), want)
    assert rel(dbr.cpu() - 0.5, want.sum(dim=(0, 2, 3))) < 1e-5
    # head backward (NHWC dx, accumulated FP32 dw and db)
    gh = t.randn((n, 3, h, w), generator=g)
    dxh = t.zeros((n, h, w, c), dtype=t.bfloat16, device="cuda")
    dwh = t.full((3, c), 0.5, device="cuda")
    dbh = t.full((3,), 0.25, device="cuda")
    assert lib.unet_head_bwd(vp(xb, 8), xb.shape[-1], c, vp(whc), vp(gh.cuda()), 3, n, h * w, vp(dxh), c, vp(dwh),
                             vp(dbh), s) == 0
    xr = x.clone().requires_grad_(True)
    wr = wh.double().requires_grad_(True)
    brh = t.zeros(3, dtype=t.float64, requires_grad=True)
    (F.conv2d(xr, wr, brh) * gh.double()).sum().backward()
    assert rel(dxh.permute(0, 3, 1, 2).float().cpu(), xr.grad) < 1e-2
    assert rel(dwh.cpu() - 0.5, wr.grad.reshape(3, c)) < 1e-4
    assert rel(dbh.cpu() - 0.25, brh.grad) < 1e-4


@pytest.mark.parametrize("c", [32, 96, 256])
def test_relu_backward_and_bias_gradient(env, c):
    """ReLU backward with the fused bias gradient over a 2 x 32 x 256 image:
    8-channel groups per pixel of 4, 12 (not a power of two) and 32."""
    t, surrogate, lib = env
    g = t.Generator().manual_seed(c)
    n, h, w = 2, 32, 256
    s = ctypes.c_void_p(t.cuda.current_stream().cuda_stream)
    yv = t.randn((n, c, h, w), generator=g).to(t.bfloat16).double()
    gv = t.randn((n, c, h, w), generator=g).to(t.bfloat16).double()
    yb, gb = nhwc_buffer(t, yv, 8, 0), nhwc_buffer(t, gv, 16, 8)
    db = t.full((c,), 0.25, device="cuda")
    assert lib.unet_relu_bwd(vp(yb), yb.shape[-1], vp(gb, 8), gb.shape[-1], c, n * h * w, vp(db), s) == 0
    want = t.where(yv > 0, gv, t.zeros_like(gv))
    assert t.equal(gb[..., 8:8 + c].permute(0, 3, 1, 2).double().cpu(), want)
    assert rel(db.cpu() - 0.25, want.sum(dim=(0, 2, 3))) < 1e-5


def test_network_matches_reference(env):
    """Whole forward pass, loss and every layer's gradients vs the FP64
    reference with the same (BF16-rounded) weights and inputs."""
    t, surrogate, lib = env
    from oracle import unet_oracle as U
    net = surrogate.UNet(batch=2, height=32, width=256, seed=4)
    # round the master weights to BF16 values so both sides use the same weights
    wts = {}
    for k, (w, b) in net.weights().items():
        wts[k] = (t.as_tensor(w).to(t.bfloat16).float().numpy(), b + 0.01)
    net.set_weights(wts)
    g = t.Generator().manual_seed(5)
    x = t.randn((2, 3, 32, 256), generator=g).to(t.bfloat16).float()
    target = t.randn((2, 3, 32, 256), generator=g)
    wc = [1.0, 0.5, 0.25]
    out = net.forward(x.cuda())
    loss = net.loss_backward(target.cuda(), wc)
    net.check_tensor_cores()
    ref_params = {k: (t.as_tensor(w, dtype=t.float64), t.as_tensor(b, dtype=t.float64)) for k, (w, b) in wts.items()}
    ref_out = U.forward(ref_params, x.double())
    assert rel(out.cpu(), ref_out) < 3e-2
    ref_loss, ref_grads = U.loss_and_grads(ref_params, x, target, t.tensor(wc))
    assert loss == pytest.approx(ref_loss, rel=3e-2)
    for name, (gw, gb) in ref_grads.items():
        p = net.params[name]
        assert rel(p["gw"].cpu(), gw) < 8e-2, name
        assert rel(p["gb"].cpu(), gb) < 8e-2, name


def test_training_reduces_loss(env):
    """Fit a smooth synthetic map from the input planes for 60 Adam steps."""
    t, surrogate, lib = env
    net = surrogate.UNet(batch=4, height=32, width=256, seed=1)
    g = t.Generator().manual_seed(9)
    y, x = t.meshgrid(t.arange(32.0), t.arange(256.0), indexing="ij")
    masks = (t.rand((4, 32, 256), generator=g) < 0.1).float()
    levels = t.tensor([0, 5, 10, 15])
    fills = t.tensor([0.5, 0.6, 0.7, 0.8])
    planes = net.planes(masks.numpy(), levels.numpy(), fills.numpy())
    target = t.stack([t.sin(2 * np.pi * x / 256)[None].expand(4, -1, -1) * fills[:, None, None],
                      (y / 32)[None].expand(4, -1, -1) * levels[:, None, None] / 15,
                      -masks], dim=1).float().cuda()
    losses = []
    for it in range(60):
        net.forward(planes)
        losses.append(net.loss_backward(target, [1.0, 1.0, 1.0]))
        net.adam(lr=2e-3)
    net.check_tensor_cores()
    assert losses[-1] < 0.2 * losses[0], (losses[0], losses[-1])


def test_graph_training_equals_step_by_step(env):
    """surrogate.train with one captured CUDA graph per step against the same
    steps launched one by one (Adam's step count and learning rate read from
    device memory in the graph). The weight and bias gradients sum over
    pixels with FP32 atomics in no fixed order, so two runs of either kind
    differ in the last bits, which Adam's division by sqrt(v) enlarges where
    a gradient is near zero (biases): losses agree to 1e-5, weights to 1e-3
    and biases to 5e-3 (relative L2)."""
    t, surrogate, lib = env
    g = t.Generator().manual_seed(5)
    planes = t.rand((8, surrogate.IN_CH, 32, 256), generator=g).cuda()
    targets = t.randn((8, surrogate.OUT_CH, 32, 256), generator=g).cuda()
    nets, hist = [], []
    for graph in (False, True):
        net = surrogate.UNet(batch=4, height=32, width=256, seed=3)
        hist.append(surrogate.train(net, planes, targets, epochs=3, lr=2e-3, seed=11, graph=graph))
        net.check_tensor_cores()
        nets.append(net)
    assert hist[0][0] == pytest.approx(hist[1][0], rel=1e-6)  # the first step's loss precedes any update
    assert hist[0] == pytest.approx(hist[1], rel=1e-5)
    assert nets[0].step_count == nets[1].step_count == 6
    for name in nets[0].params:
        for k, bound in (("w", 1e-3), ("b", 5e-3)):
            assert rel(nets[1].params[name][k].cpu(), nets[0].params[name][k].cpu()) < bound, (name, k)


def test_warm_fields_kernel(env):
    """Decode, clamp, mask and per-domain mass rescale of the warm-start
    fields against the same steps in FP64 on the host."""
    t, surrogate, lib = env
    net = surrogate.UNet(batch=2, height=32, width=256, seed=2)
    net.norm = dict(rho_mean=1.5, rho_std=0.7, u_scale=0.05)
    g = t.Generator().manual_seed(11)
    n = 3
    planes = t.rand((n, 3, 32, 256), generator=g).cuda()
    masks = (t.rand((n, 32, 256), generator=g) < 0.2).numpy().astype(np.uint8)
    mass = [1000.0, 2000.0, 3000.0]
    lo, hi = 0.03, 3.0
    out = net.warm_fields(planes, masks, mass, (lo, hi)).cpu().double()
    raw = net.predict_raw(planes).cpu().double()
    fluid = t.as_tensor(masks == 0)
    rho = t.where(fluid, (raw[:, 0] * 0.7 + 1.5).clamp(lo, hi), t.zeros(()).double())
    rho = rho * (t.tensor(mass, dtype=t.float64) / rho.sum(dim=(1, 2)))[:, None, None]
    assert t.allclose(out[:, 0], rho, rtol=1e-6, atol=1e-9)
    assert t.allclose(out[:, 1], t.where(fluid, raw[:, 1] * 0.05, t.zeros(()).double()), rtol=1e-6, atol=1e-9)
    assert t.allclose(out[:, 2], t.where(fluid, raw[:, 2] * 0.05, t.zeros(()).double()), rtol=1e-6, atol=1e-9)
    assert out[:, 0].sum(dim=(1, 2)).tolist() == pytest.approx(mass, rel=1e-12)
