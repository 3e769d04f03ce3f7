"""Plain FP64 numpy reference of the warm-start network's layers.

TEST INFRASTRUCTURE ONLY (imported by tests/ and __graft_entry__.smoke()).
The paper has no network; these are the textbook definitions of the layers
the CUDA kernels implement, written out directly (NHWC layout):

* conv3x3 "same": y[b,h,w,o] = sum_{ky,kx,c} x[b,h+ky-1,w+kx-1,c] W[o,ky,kx,c]
  (+ bias, ReLU), zero padding;
* its weight gradient dW[o,ky,kx,c] = sum_{b,h,w} dy[b,h,w,o] x[b,h+ky-1,w+kx-1,c]
  and data gradient dx[b,h,w,c] = sum dy[b,h-ky+1,w-kx+1,o] W[o,ky,kx,c];
* 2x2 max pooling, nearest 2x upsampling, channel concatenation and their
  adjoints; the masked mean-squared error.

`unet_forward` / `unet_backward` compose them into the same 4-level U-Net
as paper_2603_00035_gb300.unet (layer list below), for gradient checks.
"""
from __future__ import annotations

import numpy as np


def conv3x3(x, w, b=None, relu=False):
    x = np.asarray(x, np.float64)
    w = np.asarray(w, np.float64)
    B, H, W, C = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (0, 0)))
    y = np.zeros((B, H, W, w.shape[0]))
    for ky in range(3):
        for kx in range(3):
            y += np.einsum("bhwc,oc->bhwo", xp[:, ky:ky + H, kx:kx + W, :], w[:, ky, kx, :])
    if b is not None:
        y += np.asarray(b, np.float64)
    return np.maximum(y, 0.0) if relu else y


def conv3x3_wgrad(x, dy):
    x = np.asarray(x, np.float64)
    dy = np.asarray(dy, np.float64)
    B, H, W, C = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (0, 0)))
    dw = np.zeros((dy.shape[3], 3, 3, C))
    for ky in range(3):
        for kx in range(3):
            dw[:, ky, kx, :] = np.einsum("bhwo,bhwc->oc", dy, xp[:, ky:ky + H, kx:kx + W, :])
    return dw


def conv3x3_dgrad(dy, w):
    dy = np.asarray(dy, np.float64)
    w = np.asarray(w, np.float64)
    B, H, W, O = dy.shape
    dyp = np.pad(dy, ((0, 0), (1, 1), (1, 1), (0, 0)))
    dx = np.zeros((B, H, W, w.shape[3]))
    for ky in range(3):
        for kx in range(3):
            dx += np.einsum("bhwo,oc->bhwc", dyp[:, 2 - ky:2 - ky + H, 2 - kx:2 - kx + W, :], w[:, ky, kx, :])
    return dx


def maxpool2(x):
    B, H, W, C = x.shape
    r = np.asarray(x, np.float64).reshape(B, H // 2, 2, W // 2, 2, C).transpose(0, 1, 3, 2, 4, 5)
    r = r.reshape(B, H // 2, W // 2, 4, C)
    arg = np.argmax(r, axis=3)
    return np.take_along_axis(r, arg[:, :, :, None, :], axis=3)[:, :, :, 0, :], arg


def maxpool2_backward(dy, arg, H, W):
    B, Ho, Wo, C = dy.shape
    d = np.zeros((B, Ho, Wo, 4, C))
    np.put_along_axis(d, arg[:, :, :, None, :], np.asarray(dy, np.float64)[:, :, :, None, :], axis=3)
    d = d.reshape(B, Ho, Wo, 2, 2, C).transpose(0, 1, 3, 2, 4, 5)
    return d.reshape(B, H, W, C)


def upsample2(x):
    return np.repeat(np.repeat(np.asarray(x, np.float64), 2, axis=1), 2, axis=2)


def upsample2_backward(dy):
    B, H2, W2, C = dy.shape
    return np.asarray(dy, np.float64).reshape(B, H2 // 2, 2, W2 // 2, 2, C).sum(axis=(2, 4))


def mse(pred, target, mask, count):
    d = (np.asarray(pred, np.float64) - target) * mask
    return float((d * d).sum() / count), 2.0 * d / count


# ---- the network ---------------------------------------------------------------
# (name, Cin, Cout, relu); "pool"/"up"/"cat:<skip>" are the structural steps
def layer_plan(cin=16, base=32, cout=16):
    c = [base, 2 * base, 4 * base, 8 * base]
    return [
        ("e0a", cin, c[0], True), ("e0b", c[0], c[0], True), "skip0", "pool",
        ("e1a", c[0], c[1], True), ("e1b", c[1], c[1], True), "skip1", "pool",
        ("e2a", c[1], c[2], True), ("e2b", c[2], c[2], True), "skip2", "pool",
        ("e3a", c[2], c[3], True), ("e3b", c[3], c[3], True),
        "up", "cat:skip2", ("d2a", c[3] + c[2], c[2], True), ("d2b", c[2], c[2], True),
        "up", "cat:skip1", ("d1a", c[2] + c[1], c[1], True), ("d1b", c[1], c[1], True),
        "up", "cat:skip0", ("d0a", c[1] + c[0], c[0], True), ("d0b", c[0], c[0], True),
        ("out", c[0], cout, False),
    ]


def _ident(a):
    return a


def round_bf16(a):
    """Round to the nearest BF16 value (ties to even), returned as float64:
    the precision in which the CUDA kernels store activations and
    gradients between layers."""
    f = np.asarray(a, np.float32)
    bits = f.view(np.uint32).astype(np.uint64)
    bits = ((bits + 0x7FFF + ((bits >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return bits.view(np.float32).astype(np.float64)


def unet_forward(params, x, plan, rnd=_ident):
    """params: name -> (W [Cout,3,3,Cin], b [Cout]).  Returns (y, tape).
    rnd rounds every layer output (identity by default; round_bf16 to take
    the same precision decisions as the BF16 kernels)."""
    tape = []
    skips = {}
    last_skip = None
    h = np.asarray(x, np.float64)
    for step in plan:
        if step == "pool":
            y, arg = maxpool2(h)
            tape.append(("pool", h.shape, arg, last_skip))
            h = y
        elif step == "up":
            tape.append(("up",))
            h = upsample2(h)
        elif isinstance(step, str) and step.startswith("skip"):
            skips[step] = h
            last_skip = step
        elif isinstance(step, str) and step.startswith("cat:"):
            tape.append(("cat", h.shape[3], step[4:]))
            h = np.concatenate([h, skips[step[4:]]], axis=3)
        else:
            name, ci, co, relu = step
            W, b = params[name]
            y = rnd(conv3x3(h, W, b, relu))
            tape.append(("conv", name, h, y, relu))
            h = y
    return h, tape


def unet_backward(params, tape, dy, rnd=_ident):
    """Gradients {name: (dW, db)} of sum(dy * y) through the recorded tape
    (rnd: as in unet_forward, applied to every propagated gradient)."""
    grads = {}
    skip_grads = {}
    g = np.asarray(dy, np.float64)
    for rec in reversed(tape):
        kind = rec[0]
        if kind == "conv":
            _, name, xin, y, relu = rec
            if relu:
                g = g * (y > 0)
            W, b = params[name]
            grads[name] = (conv3x3_wgrad(xin, g), g.sum(axis=(0, 1, 2)))
            g = rnd(conv3x3_dgrad(g, W))
        elif kind == "cat":
            _, ca, sname = rec
            skip_grads[sname] = g[..., ca:]
            g = g[..., :ca]
        elif kind == "up":
            g = rnd(upsample2_backward(g))
        elif kind == "pool":
            _, shape, arg, sname = rec
            # the tensor before the pool was also saved as a skip
            g = rnd(maxpool2_backward(g, arg, shape[1], shape[2]) + skip_grads.get(sname, 0.0))
    return grads
