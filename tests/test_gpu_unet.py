"""The warm-start network's CUDA kernels (rf_unet_*) against the FP64
reference in oracle/unet_ref.py (itself pinned to scipy and finite
differences).  Inputs are BF16-representable, so the comparison isolates
the kernels' FP32 accumulation (tight) except where a kernel rounds its
output to BF16 (loose, stated per test)."""
import ctypes

import numpy as np
import pytest

from gpu_util import require_gpu, torch
from oracle import unet_ref as U
from paper_2603_00035_gb300 import _lib as L
from paper_2603_00035_gb300.api import Context, _ptr, _stream
from paper_2603_00035_gb300.unet import UNet

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def bf16(a):
    t = torch.as_tensor(np.asarray(a, np.float32)).to(torch.bfloat16)
    return t.cuda(), t.float().numpy().astype(np.float64)


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-30))


@pytest.mark.parametrize("B,H,W,Cin,Cout,relu", [(2, 13, 37, 32, 48, 1), (1, 8, 16, 16, 16, 0), (1, 24, 40, 96, 32, 1)])
def test_conv3x3_forward_dgrad_wgrad(B, H, W, Cin, Cout, relu):
    rng = np.random.default_rng(B * 100 + H)
    ctx, lib, s = Context.get(0), L.load(), _stream()
    x_t, x = bf16(rng.standard_normal((B, H, W, Cin)))
    w_t, w = bf16(rng.standard_normal((Cout, 3, 3, Cin)) * 0.2)
    bias = rng.standard_normal(Cout).astype(np.float32)
    b_t = torch.from_numpy(bias).cuda()
    y = torch.empty((B, H, W, Cout), dtype=torch.bfloat16, device="cuda")
    y32 = torch.empty((B, H, W, Cout), dtype=torch.float32, device="cuda")
    L.check(lib.rf_unet_conv3x3(ctx.handle, _ptr(x_t), B, H, W, Cin, _ptr(w_t), _ptr(b_t), Cout, relu, _ptr(y),
                                _ptr(y32), s), "conv")
    ref = U.conv3x3(x, w, bias, bool(relu))
    assert rel(y32.cpu().numpy(), ref) < 1e-5
    assert rel(y.float().cpu().numpy(), ref) < 1e-2  # BF16 output rounding
    # data gradient through the flipped weights
    dy_t, dy = bf16(rng.standard_normal((B, H, W, Cout)))
    wt = torch.empty((Cin, 3, 3, Cout), dtype=torch.bfloat16, device="cuda")
    L.check(lib.rf_unet_flip_weights(ctx.handle, _ptr(w_t), Cin, Cout, _ptr(wt), s), "flip")
    dx = torch.empty((B, H, W, Cin), dtype=torch.bfloat16, device="cuda")
    dx32 = torch.empty((B, H, W, Cin), dtype=torch.float32, device="cuda")
    L.check(lib.rf_unet_conv3x3(ctx.handle, _ptr(dy_t), B, H, W, Cout, _ptr(wt), None, Cin, 0, _ptr(dx), _ptr(dx32),
                                s), "dgrad")
    assert rel(dx32.cpu().numpy(), U.conv3x3_dgrad(dy, w)) < 1e-5
    # weight and bias gradients (FP32 accumulation into zeroed buffers)
    dw = torch.zeros((Cout, 3, 3, Cin), dtype=torch.float32, device="cuda")
    L.check(lib.rf_unet_conv3x3_wgrad(ctx.handle, _ptr(x_t), _ptr(dy_t), B, H, W, Cin, Cout, _ptr(dw), s), "wgrad")
    assert rel(dw.cpu().numpy(), U.conv3x3_wgrad(x, dy)) < 1e-5
    db = torch.zeros(Cout, dtype=torch.float32, device="cuda")
    L.check(lib.rf_unet_bias_grad(ctx.handle, _ptr(dy_t), B * H * W, Cout, _ptr(db), s), "bias_grad")
    assert rel(db.cpu().numpy(), dy.sum(axis=(0, 1, 2))) < 1e-5


@pytest.mark.parametrize("B,H,W,Cin,Cout,relu", [(2, 13, 37, 32, 48, 1), (1, 8, 16, 16, 16, 0), (1, 24, 40, 96, 32, 1),
                                               (1, 16, 32, 64, 64, 1), (2, 9, 20, 128, 64, 0), (1, 8, 16, 384, 128, 1),
                                               (2, 4, 4, 128, 256, 1), (2, 4, 6, 256, 128, 0),
                                               (8, 32, 256, 16, 32, 1), (4, 64, 192, 16, 128, 0),
                                               (2, 16, 48, 64, 192, 1), (8, 64, 160, 64, 128, 0)])
def test_conv3x3_tcgen05_forward_and_dgrad(B, H, W, Cin, Cout, relu):
    """The tcgen05 convolution (BF16 operands in shared memory, FP32
    accumulator in tensor memory) against the FP64 reference, forward and
    data gradient, and against the mma.sync kernel.  In the larger shapes
    some CTAs of the persistent kernel take several units, so they
    alternate their two accumulators and wait for the epilogue to release
    them (the last one three units).  Layers with 64 or more input and
    output channels take their weight stages from the packed copy by one
    bulk copy each, the others by tensor copies."""
    rng = np.random.default_rng(B * 1000 + H * 10 + Cin)
    ctx, lib, s = Context.get(0), L.load(), _stream()
    x_t, x = bf16(rng.standard_normal((B, H, W, Cin)))
    w_t, w = bf16(rng.standard_normal((Cout, 3, 3, Cin)) * 0.2)
    bias = rng.standard_normal(Cout).astype(np.float32)
    b_t = torch.from_numpy(bias).cuda()
    y = torch.empty((B, H, W, Cout), dtype=torch.bfloat16, device="cuda")
    y32 = torch.empty((B, H, W, Cout), dtype=torch.float32, device="cuda")
    L.check(lib.rf_unet_conv3x3_tc(ctx.handle, _ptr(x_t), B, H, W, Cin, _ptr(w_t), _ptr(b_t), Cout, relu, _ptr(y),
                                   _ptr(y32), s), "conv_tc")
    torch.cuda.synchronize()
    assert ctx.stats()["status"] == 0
    ref = U.conv3x3(x, w, bias, bool(relu))
    assert rel(y32.cpu().numpy(), ref) < 1e-5
    assert rel(y.float().cpu().numpy(), ref) < 1e-2
    y32m = torch.empty_like(y32)
    ym = torch.empty_like(y)
    L.check(lib.rf_unet_conv3x3(ctx.handle, _ptr(x_t), B, H, W, Cin, _ptr(w_t), _ptr(b_t), Cout, relu, _ptr(ym),
                                _ptr(y32m), s), "conv")
    assert (y32 - y32m).abs().max().item() <= 1e-4 * max(1.0, y32m.abs().max().item())
    dy_t, dy = bf16(rng.standard_normal((B, H, W, Cout)))
    wt = torch.empty((Cin, 3, 3, Cout), dtype=torch.bfloat16, device="cuda")
    L.check(lib.rf_unet_flip_weights(ctx.handle, _ptr(w_t), Cin, Cout, _ptr(wt), s), "flip")
    dx = torch.empty((B, H, W, Cin), dtype=torch.bfloat16, device="cuda")
    dx32 = torch.empty((B, H, W, Cin), dtype=torch.float32, device="cuda")
    L.check(lib.rf_unet_conv3x3_tc(ctx.handle, _ptr(dy_t), B, H, W, Cout, _ptr(wt), None, Cin, 0, _ptr(dx),
                                   _ptr(dx32), s), "dgrad_tc")
    assert rel(dx32.cpu().numpy(), U.conv3x3_dgrad(dy, w)) < 1e-5


@pytest.mark.parametrize("B,H,W,Cin,Cout", [(1, 8, 16, 16, 16), (2, 13, 37, 32, 48), (1, 24, 70, 96, 32),
                                            (2, 9, 130, 64, 128), (1, 6, 20, 384, 128), (2, 4, 6, 256, 256),
                                            (3, 5, 64, 48, 144)])
def test_conv3x3_wgrad_tcgen05(B, H, W, Cin, Cout):
    """The tcgen05 weight gradient (MN-major BF16 operands, FP32 accumulators
    in tensor memory, split over pixel rows) against the FP64 reference and
    the mma.sync kernel: ragged widths (several 64-pixel segments and a
    partial one), output channels beyond a 128 tile, Cin not a multiple of
    32 (16-channel tiles)."""
    rng = np.random.default_rng(B * 7 + H * 3 + Cin)
    ctx, lib, s = Context.get(0), L.load(), _stream()
    x_t, x = bf16(rng.standard_normal((B, H, W, Cin)))
    dy_t, dy = bf16(rng.standard_normal((B, H, W, Cout)))
    dw = torch.zeros((Cout, 3, 3, Cin), dtype=torch.float32, device="cuda")
    L.check(lib.rf_unet_conv3x3_wgrad_tc(ctx.handle, _ptr(x_t), _ptr(dy_t), B, H, W, Cin, Cout, _ptr(dw), s),
            "wgrad_tc")
    torch.cuda.synchronize()
    assert ctx.stats()["status"] == 0
    ref = U.conv3x3_wgrad(x, dy)
    assert rel(dw.cpu().numpy(), ref) < 1e-5
    dwm = torch.zeros_like(dw)
    L.check(lib.rf_unet_conv3x3_wgrad(ctx.handle, _ptr(x_t), _ptr(dy_t), B, H, W, Cin, Cout, _ptr(dwm), s), "wgrad")
    assert (dw - dwm).abs().max().item() <= 1e-4 * max(1.0, dwm.abs().max().item())


def test_pool_upsample_concat_relu_mse():
    rng = np.random.default_rng(7)
    ctx, lib, s = Context.get(0), L.load(), _stream()
    B, H, W, C = 2, 10, 14, 16
    x_t, x = bf16(rng.standard_normal((B, H, W, C)))
    y = torch.empty((B, H // 2, W // 2, C), dtype=torch.bfloat16, device="cuda")
    arg = torch.empty(y.shape, dtype=torch.uint8, device="cuda")
    L.check(lib.rf_unet_maxpool2(ctx.handle, _ptr(x_t), B, H, W, C, _ptr(y), _ptr(arg), s), "pool")
    ry, rarg = U.maxpool2(x)
    assert np.array_equal(y.float().cpu().numpy(), ry)
    dy_t, dy = bf16(rng.standard_normal(ry.shape))
    dx = torch.empty_like(x_t)
    L.check(lib.rf_unet_maxpool2_backward(ctx.handle, _ptr(dy_t), _ptr(arg), B, H, W, C, _ptr(dx), s), "pool_bwd")
    assert np.array_equal(dx.float().cpu().numpy(), U.maxpool2_backward(dy, rarg, H, W))
    up = torch.empty((B, 2 * H, 2 * W, C), dtype=torch.bfloat16, device="cuda")
    L.check(lib.rf_unet_upsample2(ctx.handle, _ptr(x_t), B, H, W, C, _ptr(up), s), "up")
    assert np.array_equal(up.float().cpu().numpy(), U.upsample2(x))
    du_t, du = bf16(rng.standard_normal((B, 2 * H, 2 * W, C)))
    dd = torch.empty_like(x_t)
    L.check(lib.rf_unet_upsample2_backward(ctx.handle, _ptr(du_t), B, H, W, C, _ptr(dd), s), "up_bwd")
    assert rel(dd.float().cpu().numpy(), U.upsample2_backward(du)) < 1e-2
    # concat / split
    a_t, a = bf16(rng.standard_normal((B, H, W, 16)))
    c_t, c = bf16(rng.standard_normal((B, H, W, 32)))
    cat = torch.empty((B, H, W, 48), dtype=torch.bfloat16, device="cuda")
    L.check(lib.rf_unet_concat(ctx.handle, _ptr(a_t), 16, _ptr(c_t), 32, B * H * W, _ptr(cat), 0, s), "cat")
    assert np.array_equal(cat.float().cpu().numpy(), np.concatenate([a, c], axis=3))
    a2, c2 = torch.empty_like(a_t), torch.empty_like(c_t)
    L.check(lib.rf_unet_concat(ctx.handle, _ptr(a2), 16, _ptr(c2), 32, B * H * W, _ptr(cat), 1, s), "split")
    assert torch.equal(a2, a_t) and torch.equal(c2, c_t)
    # relu backward
    g = dy_t.clone()
    L.check(lib.rf_unet_relu_backward(ctx.handle, _ptr(g), _ptr(y), g.numel(), s), "relu_bwd")
    assert np.array_equal(g.float().cpu().numpy(), dy * (ry > 0))
    # masked MSE on channel 0
    pred = torch.from_numpy(rng.standard_normal((B, H, W, C)).astype(np.float32)).cuda()
    tgt = torch.from_numpy(rng.standard_normal((B, H, W)).astype(np.float32)).cuda()
    mask = torch.from_numpy((rng.random((B, H, W)) < 0.5).astype(np.float32)).cuda()
    loss = torch.zeros(1, device="cuda")
    dp = torch.empty((B, H, W, C), dtype=torch.bfloat16, device="cuda")
    cnt = float(mask.sum())
    L.check(lib.rf_unet_mse(ctx.handle, _ptr(pred), C, _ptr(tgt), _ptr(mask), B * H * W, cnt, _ptr(dp), _ptr(loss),
                            s), "mse")
    rl, rg = U.mse(pred.cpu().numpy()[..., 0], tgt.cpu().numpy(), mask.cpu().numpy(), cnt)
    assert float(loss) == pytest.approx(rl, rel=1e-5)
    assert rel(dp.float().cpu().numpy()[..., 0], rg) < 1e-2
    assert float(dp.float()[..., 1:].abs().max()) == 0.0


def test_unet_gradients_match_reference():
    """Whole network: forward output and every weight/bias gradient vs the
    FP64 reference evaluated with the same BF16 weights and input, rounding
    activations and gradients to BF16 at the same points as the kernels (so
    both sides take the same ReLU decisions); what remains is FP32 vs FP64
    accumulation and the odd rounding-boundary case."""
    net = UNet(cin=16, base=32, cout=16, seed=1)
    rng = np.random.default_rng(3)
    x_t, x = bf16(rng.standard_normal((1, 32, 32, 16)))
    out = net.forward(x_t)
    params = {k: (net.Wbf[k].float().cpu().numpy().astype(np.float64), net.b[k].cpu().numpy().astype(np.float64))
              for k in net.W}
    plan = U.layer_plan(16, 32, 16)
    ref, tape = U.unet_forward(params, x, plan, rnd=U.round_bf16)
    assert rel(out.cpu().numpy(), ref) < 1e-2
    dy_t, dy = bf16(rng.standard_normal(ref.shape) * 0.1)
    net.zero_grad()
    net.backward(dy_t)
    grads = U.unet_backward(params, tape, dy, rnd=U.round_bf16)
    # one-ulp BF16 re-roundings after FP32-vs-FP64 accumulation differences
    # flip a few ReLU masks, which spread through ~25 backward layers: check
    # direction tightly and magnitude loosely (each kernel is pinned to 1e-5
    # by the per-layer tests above)
    def cos(a, b):
        a = np.asarray(a, np.float64).ravel()
        b = np.asarray(b, np.float64).ravel()
        return float(a @ b / (np.linalg.norm(a) * np.linalg.norm(b)))
    for k in net.W:
        gw, gb = net.gW[k].cpu().numpy(), net.gb[k].cpu().numpy()
        assert cos(gw, grads[k][0]) > 0.99, (k, cos(gw, grads[k][0]))
        assert rel(gw, grads[k][0]) < 0.15, (k, rel(gw, grads[k][0]))
        assert rel(gb, grads[k][1]) < 0.15, (k, rel(gb, grads[k][1]))


@pytest.mark.parametrize("B,H,W,seed", [(1, 32, 32, 3), (2, 16, 40, 4)])
def test_unet_integer_network_bit_exact(B, H, W, seed):
    """Whole network, bit for bit.  Weights in {-1, 0, 1} (about three
    non-zeros per output channel and input position), integer biases, input
    and output gradient: every stored activation and gradient is an integer
    and every product and partial sum is an integer far below 2^24 (at most
    a few 10^5 for these seeds, the weight-gradient sums over all pixels),
    so FP32 accumulation in any order is exact, FP64 agrees, and both sides
    round to BF16 identically (values above 256 do get rounded, to even
    integers).  The forward output and every weight and bias gradient must
    then equal the FP64 reference exactly: a wrong skip, concat split,
    pooling route, upsample sum or ReLU mask anywhere in the composed
    network shows as a mismatch, with no accumulation noise to hide it."""
    net = UNet(cin=16, base=32, cout=16, seed=0)
    rng = np.random.default_rng(seed)
    params = {}
    for step in net.plan:
        if isinstance(step, tuple):
            name, ci, co, relu = step
            nz = rng.random((co, 3, 3, ci)) < 3.0 / (9 * ci)
            w = np.where(nz, rng.choice([-1.0, 1.0], size=nz.shape), 0.0)
            b = rng.integers(-1, 3, size=co).astype(np.float64) if relu else np.zeros(co)
            net.W[name].copy_(torch.from_numpy(w.astype(np.float32)))
            net.b[name].copy_(torch.from_numpy(b.astype(np.float32)))
            params[name] = (w, b)
    net.refresh()
    x_t, x = bf16(rng.integers(-3, 4, size=(B, H, W, 16)))
    out = net.forward(x_t)
    ref, tape = U.unet_forward(params, x, net.plan, rnd=U.round_bf16)
    # the kernel returns the last layer's FP32 sum, before any BF16 rounding
    last = tape[-1]
    assert last[0] == "conv" and last[1] == "out"
    ref_out = U.conv3x3(last[2], params["out"][0], params["out"][1], False)
    np.testing.assert_array_equal(out.cpu().numpy(), ref_out)
    dy_t, dy = bf16(rng.integers(-2, 3, size=ref.shape))
    net.zero_grad()
    net.backward(dy_t)
    grads = U.unet_backward(params, tape, dy, rnd=U.round_bf16)
    for k in net.W:
        gw, gb = grads[k]
        # the case is not degenerate: gradient reaches every layer
        assert (gw != 0).mean() > 0.02 and (gb != 0).any(), k
        np.testing.assert_array_equal(net.gW[k].cpu().numpy(), gw, err_msg=k)
        np.testing.assert_array_equal(net.gb[k].cpu().numpy(), gb, err_msg=k)


def test_unet_training_reduces_loss():
    net = UNet(seed=2)
    opt = torch.optim.Adam(net.parameters(), lr=2e-3)
    rng = np.random.default_rng(4)
    x_t, _ = bf16(rng.standard_normal((2, 32, 32, 16)))
    # a smooth target that depends on the input
    tgt = torch.tanh(x_t.float()[..., 0] + 0.5 * x_t.float()[..., 1]).contiguous()
    losses = []
    for it in range(30):
        out = net.forward(x_t)
        loss, dout = net.mse(out, tgt)
        net.zero_grad()
        net.backward(dout)
        net.attach_grads()
        opt.step()
        net.refresh()
        losses.append(float(loss))
    assert losses[-1] < 0.5 * losses[0], losses[::5]
