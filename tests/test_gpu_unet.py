"""U-Net kernels and network against the CPU reference (oracle/unet_oracle).

BF16 storage with FP32 sums: the reference gets the same BF16-rounded
weights and inputs in FP64, so the remaining differences are accumulation
order and the BF16 rounding of intermediate activations and gradients.
Bounds: single kernels 1e-2 relative (L2) of the output; the whole network's
output 3e-2 and every layer's weight gradient 8e-2 relative (L2) after the
16 layers of BF16 round trips.
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
    return torch, surrogate, lib


def rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def bf(t, x):
    return x.to(t.bfloat16)


def ref_conv(t, x, w, b=None):
    import torch.nn.functional as F
    xp = F.pad(F.pad(x, (1, 1, 0, 0), mode="circular"), (0, 0, 1, 1))
    return F.conv2d(xp, w, b)


@pytest.mark.parametrize("ci,co,h,w", [(3, 32, 64, 256), (96, 32, 32, 64), (256, 128, 8, 32)])
def test_conv3x3_forward_backward(env, ci, co, h, w):
    t, surrogate, lib = env
    g = t.Generator().manual_seed(ci + co)
    n = 2
    x = t.randn((n, ci, h, w), generator=g)
    wt = t.randn((co, ci, 3, 3), generator=g) * (2.0 / (9 * ci)) ** 0.5
    b = t.randn(co, generator=g) * 0.1
    dy = t.randn((n, co, h, w), generator=g)
    xb, wb, dyb = bf(t, x).cuda(), bf(t, wt).cuda(), bf(t, dy).cuda()
    s = ctypes.c_void_p(t.cuda.current_stream().cuda_stream)
    y = t.empty((n, co, h, w), dtype=t.bfloat16, device="cuda")
    bias = b.float().cuda()
    assert lib.unet_conv3x3_fwd(ctypes.c_void_p(xb.data_ptr()), ci, ci * h * w, ctypes.c_void_p(wb.data_ptr()),
                                ctypes.c_void_p(bias.data_ptr()), ctypes.c_void_p(y.data_ptr()), co, co * h * w,
                                n, h, w, 1, s) == 0
    ref = t.relu(ref_conv(t, xb.double().cpu(), wb.double().cpu(), b.double()))
    assert rel(y.float().cpu(), ref) < 1e-2
    # gradient w.r.t. input (no activation) and w.r.t. weights/bias
    dx = t.empty((n, ci, h, w), dtype=t.bfloat16, device="cuda")
    assert lib.unet_conv3x3_bwd_data(ctypes.c_void_p(dyb.data_ptr()), co, co * h * w,
                                     ctypes.c_void_p(wb.data_ptr()), ctypes.c_void_p(dx.data_ptr()), ci,
                                     ci * h * w, n, h, w, s) == 0
    dw = t.zeros((co, ci, 3, 3), device="cuda")
    db = t.zeros(co, device="cuda")
    assert lib.unet_conv3x3_bwd_weight(ctypes.c_void_p(xb.data_ptr()), ci, ci * h * w,
                                       ctypes.c_void_p(dyb.data_ptr()), co, co * h * w,
                                       ctypes.c_void_p(dw.data_ptr()), ctypes.c_void_p(db.data_ptr()), n, h, w,
                                       s) == 0
    xr = xb.double().cpu().requires_grad_(True)
    wr = wb.double().cpu().requires_grad_(True)
    br = t.zeros(co, dtype=t.float64, requires_grad=True)
    (ref_conv(t, xr, wr, br) * dyb.double().cpu()).sum().backward()
    assert rel(dx.float().cpu(), xr.grad) < 1e-2
    assert rel(dw.cpu(), wr.grad) < 1e-2
    assert rel(db.cpu(), br.grad) < 1e-2


def test_pool_upsample_head(env):
    t, surrogate, lib = env
    import torch.nn.functional as F
    g = t.Generator().manual_seed(7)
    n, c, h, w = 2, 32, 16, 64
    x = bf(t, t.randn((n, c, h, w), generator=g)).cuda()
    s = ctypes.c_void_p(t.cuda.current_stream().cuda_stream)
    p = t.empty((n, c, h // 2, w // 2), dtype=t.bfloat16, device="cuda")
    lib.unet_pool2_fwd(ctypes.c_void_p(x.data_ptr()), c * h * w, ctypes.c_void_p(p.data_ptr()), c * h * w // 4,
                       c, n, h, w, s)
    assert rel(p.float().cpu(), F.avg_pool2d(x.double().cpu(), 2)) < 1e-2
    u = t.empty((n, c, h, w), dtype=t.bfloat16, device="cuda")
    lib.unet_up2_fwd(ctypes.c_void_p(p.data_ptr()), c * h * w // 4, ctypes.c_void_p(u.data_ptr()), c * h * w, c, n,
                     h // 2, w // 2, s)
    assert t.equal(u.cpu(), F.interpolate(p.cpu().float(), scale_factor=2, mode="nearest").to(t.bfloat16))
    # adjoints: <pool(x), y> = <x, pool^T(y)>, <up(a), b> = <a, up^T(b)>
    yb = bf(t, t.randn((n, c, h // 2, w // 2), generator=g)).cuda()
    dx = t.zeros((n, c, h, w), dtype=t.bfloat16, device="cuda")
    lib.unet_pool2_bwd(ctypes.c_void_p(yb.data_ptr()), c * h * w // 4, ctypes.c_void_p(dx.data_ptr()), c * h * w,
                       c, n, h, w, 0, s)
    lhs = (F.avg_pool2d(x.double().cpu(), 2) * yb.double().cpu()).sum().item()
    assert abs(lhs - (x.double().cpu() * dx.double().cpu()).sum().item()) < 2e-2 * abs(lhs) + 1e-3
    bb = bf(t, t.randn((n, c, h, w), generator=g)).cuda()
    da = t.empty((n, c, h // 2, w // 2), dtype=t.bfloat16, device="cuda")
    lib.unet_up2_bwd(ctypes.c_void_p(bb.data_ptr()), c * h * w, ctypes.c_void_p(da.data_ptr()), c * h * w // 4,
                     c, n, h // 2, w // 2, s)
    lhs = (F.interpolate(yb.double().cpu(), scale_factor=2, mode="nearest") * bb.double().cpu()).sum().item()
    assert abs(lhs - (yb.double().cpu() * da.double().cpu()).sum().item()) < 2e-2 * abs(lhs) + 1e-3
    # 1x1 head
    wh = bf(t, t.randn((3, c, 1, 1), generator=g)).cuda()
    bh = t.randn(3, generator=g).float().cuda()
    yh = t.empty((n, 3, h, w), device="cuda")
    lib.unet_head_fwd(ctypes.c_void_p(x.data_ptr()), c, c * h * w, ctypes.c_void_p(wh.data_ptr()),
                      ctypes.c_void_p(bh.data_ptr()), ctypes.c_void_p(yh.data_ptr()), 3, n, h * w, s)
    ref = F.conv2d(x.double().cpu(), wh.double().cpu(), bh.double().cpu())
    assert rel(yh.cpu(), ref) < 1e-3


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
    assert losses[-1] < 0.2 * losses[0], (losses[0], losses[-1])
