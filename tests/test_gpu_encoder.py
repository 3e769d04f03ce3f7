"""The covariate encoder's head (rf_encoder_combine and its adjoint) against
the FP64 oracle, the MLP-as-1x1-convolution pathway against dense layers,
and end-to-end training through the solver reducing the held-out error."""
import numpy as np
import pytest

from gpu_util import require_gpu, to_dev, torch
from oracle import encoder_ref as E
from oracle import unet_ref as U
from paper_2603_00035_gb300 import _lib as L
from paper_2603_00035_gb300 import api
from paper_2603_00035_gb300.api import _ptr, _stream

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


@pytest.mark.parametrize("B,H,W", [(3, 5, 7), (2, 64, 64), (1, 1, 1)])
def test_combine_and_adjoint_match_oracle(B, H, W):
    rng = np.random.default_rng(B * 100 + H)
    C = Cb = 16
    alpha = 0.7
    local = rng.standard_normal((B, H, W, C)).astype(np.float32)
    base = rng.standard_normal((B, Cb)).astype(np.float32)
    ctx, lib = api.Context.get(0), L.load()
    local_t, base_t = to_dev(local), to_dev(base)  # kept alive across the call
    gb = torch.empty((B, 5, H, W), dtype=torch.float32, device="cuda")
    L.check(lib.rf_encoder_combine(ctx.handle, _ptr(local_t), B, H, W, C, _ptr(base_t), Cb, alpha, _ptr(gb),
                                   _stream()), "combine")
    want = E.combine(local, base, alpha)
    assert np.abs(gb.cpu().numpy() - want).max() <= 1e-6 * (1 + np.abs(want).max())
    dgb = rng.standard_normal((B, 5, H, W)).astype(np.float32)
    dgb_t = to_dev(dgb)
    dl = torch.empty((B, H, W, C), dtype=torch.bfloat16, device="cuda")
    db = torch.empty((B, Cb), dtype=torch.bfloat16, device="cuda")
    L.check(lib.rf_encoder_combine_backward(ctx.handle, _ptr(dgb_t), B, H, W, C, Cb, alpha, _ptr(dl), _ptr(db),
                                            _stream()), "combine_bwd")
    wl, wb = E.combine_backward(dgb, alpha, C, Cb)
    gl, gbb = dl.float().cpu().numpy(), db.float().cpu().numpy()
    assert np.abs(gl - wl).max() <= 2 ** -8 * (np.abs(wl).max() + 1e-30)  # one BF16 rounding
    assert np.abs(gbb - wb).max() <= 2 ** -8 * np.abs(wb).max() + 1e-4 * np.abs(dgb).sum(axis=(2, 3)).max()
    assert np.all(gl[..., 5:] == 0) and np.all(gbb[:, 5:] == 0)


def test_mlp_on_a_1x1_image_is_a_dense_network():
    from paper_2603_00035_gb300.encoder import mlp_plan
    from paper_2603_00035_gb300.unet import UNet
    net = UNet(seed=3, plan=mlp_plan())
    rng = np.random.default_rng(5)
    x = rng.standard_normal((4, 1, 1, 16)).astype(np.float32)
    xt = to_dev(x).to(torch.bfloat16)
    out = net.forward(xt).cpu().numpy()[:, 0, 0, :]
    h = xt.float().cpu().numpy()[:, 0, 0, :].astype(np.float64)
    for name, _, _, relu in mlp_plan():
        w = net.Wbf[name].float().cpu().numpy().astype(np.float64)[:, 1, 1, :]  # centre tap
        h = h @ w.T + net.b[name].cpu().numpy()
        if relu:
            h = np.maximum(h, 0.0)
        if name != "out":
            h = U.round_bf16(h)  # activations are stored in BF16
    assert np.abs(out - h).max() <= 1e-2 * (1 + np.abs(h).max())


def test_encoder_training_reduces_held_out_error():
    from paper_2603_00035_gb300.encoder import train_synthetic
    r = train_synthetic(steps=120, batch=4, n=32, n_sources=2, obs_frac=0.2, seed=1, eval_batches=1, log_every=0)
    assert r["status"] == 0
    before, after = r["held_out_before"], r["held_out_after"]
    # the arrival times and the drift are learned; the spatial metric is the
    # hard part (sparse times constrain it weakly) and must not get worse
    assert after["T"] < 0.8 * before["T"], r
    assert after["b"] < 0.8 * before["b"], r
    assert after["g"] < 1.05 * before["g"], r
