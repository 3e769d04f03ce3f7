"""Plain FP64 numpy reference of the covariate encoder's head (Sec. 5,
"Encoder Architecture"): G = G0 + alpha G_local, b = b0 + alpha b_local.

TEST INFRASTRUCTURE ONLY (imported by tests/ and __graft_entry__.smoke()).

Layouts: local [B, H, W, C] (channels 0..4 = residuals of g11, g12, g22,
b1, b2), base [B, Cb] (channels 0..4 = G0, b0), gb [B, 5, H, W]."""
from __future__ import annotations

import numpy as np


def combine(local, base, alpha):
    local = np.asarray(local, np.float64)
    base = np.asarray(base, np.float64)
    return base[:, :5, None, None] + alpha * np.moveaxis(local[..., :5], -1, 1)


def combine_backward(dgb, alpha, C, Cb):
    """Adjoint of combine: (dlocal [B, H, W, C], dbase [B, Cb]), zero on the
    channels combine does not read."""
    dgb = np.asarray(dgb, np.float64)
    B, _, H, W = dgb.shape
    dlocal = np.zeros((B, H, W, C))
    dlocal[..., :5] = alpha * np.moveaxis(dgb, 1, -1)
    dbase = np.zeros((B, Cb))
    dbase[:, :5] = dgb.sum(axis=(2, 3))
    return dlocal, dbase
