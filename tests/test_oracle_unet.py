"""Pins of the FP64 reference of the warm-start network (oracle/unet_ref.py):
its convolution agrees with scipy's correlate, and its backward (data,
weight and bias gradients through pooling, upsampling, skips and ReLUs) agrees
with central finite differences of its forward."""
import numpy as np
import pytest
from scipy.signal import correlate

from oracle import unet_ref as U


def test_conv_matches_scipy_correlate():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((2, 7, 9, 3))
    w = rng.standard_normal((4, 3, 3, 3))
    y = U.conv3x3(x, w)
    for b in range(2):
        for o in range(4):
            ref = sum(correlate(x[b, :, :, c], w[o, :, :, c], mode="same") for c in range(3))
            assert np.allclose(y[b, :, :, o], ref, atol=1e-12)


def test_conv_gradients_finite_differences():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((1, 5, 6, 2))
    w = rng.standard_normal((3, 3, 3, 2))
    dy = rng.standard_normal((1, 5, 6, 3))
    f = lambda xx, ww: float((U.conv3x3(xx, ww) * dy).sum())
    dw = U.conv3x3_wgrad(x, dy)
    dx = U.conv3x3_dgrad(dy, w)
    e = 1e-6
    for idx in [(0, 0, 0, 0), (2, 1, 2, 1), (1, 2, 0, 0)]:
        wp, wm = w.copy(), w.copy()
        wp[idx] += e
        wm[idx] -= e
        assert dw[idx] == pytest.approx((f(x, wp) - f(x, wm)) / (2 * e), rel=1e-7, abs=1e-9)
    for idx in [(0, 0, 0, 0), (0, 4, 5, 1), (0, 2, 3, 0)]:
        xp, xm = x.copy(), x.copy()
        xp[idx] += e
        xm[idx] -= e
        assert dx[idx] == pytest.approx((f(xp, w) - f(xm, w)) / (2 * e), rel=1e-7, abs=1e-9)


def test_unet_backward_finite_differences():
    rng = np.random.default_rng(2)
    plan = U.layer_plan(cin=2, base=2, cout=1)
    params = {}
    for step in plan:
        if isinstance(step, tuple):
            name, ci, co, relu = step
            params[name] = (rng.standard_normal((co, 3, 3, ci)) * np.sqrt(2.0 / (9 * ci)), rng.standard_normal(co) * 0.1)
    x = rng.standard_normal((1, 16, 16, 2))
    dy = rng.standard_normal((1, 16, 16, 1))
    y, tape = U.unet_forward(params, x, plan)
    grads = U.unet_backward(params, tape, dy)
    f = lambda: float((U.unet_forward(params, x, plan)[0] * dy).sum())
    e = 1e-6
    checked = 0
    for name in ["e0a", "e1b", "e3a", "d2a", "d0a", "out"]:
        W, b = params[name]
        for idx in [(0, 1, 1, 0), (0, 0, 2, W.shape[3] - 1)]:
            orig = W[idx]
            W[idx] = orig + e
            fp = f()
            W[idx] = orig - e
            fm = f()
            W[idx] = orig
            fd = (fp - fm) / (2 * e)
            assert grads[name][0][idx] == pytest.approx(fd, rel=1e-5, abs=1e-7), name
            checked += 1
        orig = b[0]
        b[0] = orig + e
        fp = f()
        b[0] = orig - e
        fm = f()
        b[0] = orig
        assert grads[name][1][0] == pytest.approx((fp - fm) / (2 * e), rel=1e-5, abs=1e-7), name
    assert checked == 12


def test_round_bf16():
    vals = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 2.0 ** -7, 1.0 + 3 * 2.0 ** -8, -3.1415926, 0.0])
    r = U.round_bf16(vals)
    # ties to even at 1 + 2^-8; exactly representable values unchanged
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1.0 + 2.0 ** -7 and r[3] == 1.0 + 2.0 ** -6
    assert r[4] == -3.140625 and r[5] == 0.0
