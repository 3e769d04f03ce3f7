"""Pins of the encoder-head oracle: constant inputs give the closed form,
and the backward is the adjoint of the forward (<combine(x), y> equals
<x, combine_backward(y)> for random x, y)."""
import numpy as np

from oracle import encoder_ref as E


def test_constant_inputs():
    B, H, W, C, Cb = 2, 3, 4, 16, 16
    local = np.zeros((B, H, W, C))
    local[..., 1] = 2.0
    local[..., 7] = 9.0  # not read
    base = np.zeros((B, Cb))
    base[:, 0] = [1.0, 3.0]
    base[:, 9] = 5.0  # not read
    gb = E.combine(local, base, 0.5)
    assert gb.shape == (B, 5, H, W)
    assert np.all(gb[0, 0] == 1.0) and np.all(gb[1, 0] == 3.0) and np.all(gb[:, 1] == 1.0)
    assert np.all(gb[:, 2:] == 0.0)


def test_backward_is_the_adjoint():
    rng = np.random.default_rng(0)
    B, H, W, C, Cb, alpha = 3, 5, 7, 16, 16, 0.7
    local, base = rng.normal(size=(B, H, W, C)), rng.normal(size=(B, Cb))
    dgb = rng.normal(size=(B, 5, H, W))
    dl, db = E.combine_backward(dgb, alpha, C, Cb)
    lhs = float((E.combine(local, base, alpha) * dgb).sum())
    rhs = float((local * dl).sum() + (base * db).sum())
    assert abs(lhs - rhs) < 1e-10 * max(1.0, abs(lhs))
    assert np.all(dl[..., 5:] == 0) and np.all(db[:, 5:] == 0)
