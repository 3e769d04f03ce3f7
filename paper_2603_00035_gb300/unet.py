"""The learned warm start's network: a 4-level U-Net (32 base channels)
whose every convolution, pooling, upsampling, concatenation, ReLU backward
and loss runs in librf's kernels (rf_unet_*), BF16 activations with FP32
accumulation; the wide convolutions run on the tcgen05 tensor cores.  PyTorch holds the tensors and runs Adam on the FP32 master
weights.

Layers (NHWC, channels padded to multiples of 16):
  e0: 16 -> 32 -> 32 (skip0), pool;  e1: 32 -> 64 -> 64 (skip1), pool;
  e2: 64 -> 128 -> 128 (skip2), pool; e3: 128 -> 256 -> 256;
  up, cat skip2, d2: 384 -> 128 -> 128; up, cat skip1, d1: 192 -> 64 -> 64;
  up, cat skip0, d0: 96 -> 32 -> 32;  out: 32 -> 16 (channel 0 = T guess).
All convolutions are 3x3 "same" with bias; ReLU everywhere except `out`.
"""
from __future__ import annotations

import ctypes
import math

import torch

from . import _lib as L
from .api import Context, _ptr, _stream


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


def _chk(st, where):
    L.check(st, where)


def conv3x3(lib, h, x, B, H, W, Cin, w, bias, Cout, relu, y, y32, s):
    """rf_unet_conv3x3 on the tcgen05 kernel (persistent, tensor copies,
    2-4 pixel tiles sharing each weight stage, two tensor-memory accumulator
    sets) when both channel counts are at least 32 -- measured on GB300 at
    446-470 vs 236-248 TFLOP/s (128+ output channels), 268 vs 187 (64 -> 64),
    174-200 vs 169-196 (32 -> 32 / 64) -- and on the mma.sync kernel for the
    16-channel layers (159 vs 144 TFLOP/s at 16 -> 32)."""
    fn = lib.rf_unet_conv3x3_tc if (Cin >= 32 and Cout >= 32) else lib.rf_unet_conv3x3
    return fn(h, x, B, H, W, Cin, w, bias, Cout, relu, y, y32, s)


def conv3x3_wgrad(lib, h, x, dy, B, H, W, Cin, Cout, dw, s):
    """rf_unet_conv3x3_wgrad on the tcgen05 kernel for 128 or more output
    channels, where it measured faster on GB300 (153-202 vs 140-150 TFLOP/s:
    8 x 128^2 at 128 -> 128, 8 x 64^2 at 256 -> 256 and 384 -> 128), and on
    the mma.sync kernel for the narrow layers (82-130 vs 44-75 TFLOP/s at
    16-64 output channels: the tensor-core tile is 128 output channels)."""
    fn = lib.rf_unet_conv3x3_wgrad_tc if Cout % 128 == 0 else lib.rf_unet_conv3x3_wgrad
    return fn(h, x, dy, B, H, W, Cin, Cout, dw, s)


class UNet:
    def __init__(self, cin=16, base=32, cout=16, device="cuda", seed=0, ctx=None, plan=None):
        """plan: a layer list in layer_plan's format (the last convolution
        named "out"); default the 4-level U-Net."""
        self.dev = torch.device(device)
        self.ctx = ctx or Context.get(self.dev)
        self.plan = plan if plan is not None else layer_plan(cin, base, cout)
        self.cin, self.cout = cin, cout
        g = torch.Generator(device="cpu").manual_seed(seed)
        self.W, self.b = {}, {}
        for step in self.plan:
            if isinstance(step, tuple):
                name, ci, co, relu = step
                std = math.sqrt(2.0 / (9 * ci)) if relu else math.sqrt(1.0 / (9 * ci))
                self.W[name] = (torch.randn((co, 3, 3, ci), generator=g) * std).to(self.dev).requires_grad_(False)
                self.b[name] = torch.zeros(co, device=self.dev)
        self.gW = {k: torch.zeros_like(v) for k, v in self.W.items()}
        self.gb = {k: torch.zeros_like(v) for k, v in self.b.items()}
        self.Wbf = {k: torch.empty(v.shape, dtype=torch.bfloat16, device=self.dev) for k, v in self.W.items()}
        self.Wflip = {k: torch.empty((v.shape[3], 3, 3, v.shape[0]), dtype=torch.bfloat16, device=self.dev)
                      for k, v in self.W.items()}
        self.refresh()

    # ---- parameters ---------------------------------------------------------------
    def parameters(self):
        return list(self.W.values()) + list(self.b.values())

    def attach_grads(self):
        for k in self.W:
            self.W[k].grad = self.gW[k]
            self.b[k].grad = self.gb[k]

    def refresh(self):
        """BF16 copies (and flipped copies for the data gradient) of the FP32
        master weights."""
        lib, s = L.load(), _stream()
        for k, w in self.W.items():
            _chk(lib.rf_unet_cast_bf16(self.ctx.handle, _ptr(w), _ptr(self.Wbf[k]), w.numel(), s), "cast")
            co, _, _, ci = w.shape
            _chk(lib.rf_unet_flip_weights(self.ctx.handle, _ptr(self.Wbf[k]), ci, co, _ptr(self.Wflip[k]), s), "flip")

    def state_dict(self):
        return {"W": {k: v.detach().cpu() for k, v in self.W.items()},
                "b": {k: v.detach().cpu() for k, v in self.b.items()}}

    def load_state_dict(self, d):
        for k in self.W:
            self.W[k].copy_(d["W"][k])
            self.b[k].copy_(d["b"][k])
        self.refresh()

    # ---- forward ------------------------------------------------------------------
    def forward(self, x):
        """x: [B, H, W, cin] bfloat16 (H, W divisible by 8).  Returns the FP32
        output [B, H, W, cout]; activations are kept for backward()."""
        lib, s, h = L.load(), _stream(), self.ctx.handle
        B, H, W, _ = x.shape
        tape = []
        skips = {}
        last_skip = None
        cur = x.contiguous()
        out32 = None
        for step in self.plan:
            B_, H_, W_, C_ = cur.shape
            if step == "pool":
                y = torch.empty((B_, H_ // 2, W_ // 2, C_), dtype=torch.bfloat16, device=self.dev)
                arg = torch.empty(y.shape, dtype=torch.uint8, device=self.dev)
                _chk(lib.rf_unet_maxpool2(h, _ptr(cur), B_, H_, W_, C_, _ptr(y), _ptr(arg), s), "maxpool2")
                tape.append(("pool", cur.shape, arg, last_skip))
                cur = y
            elif step == "up":
                y = torch.empty((B_, 2 * H_, 2 * W_, C_), dtype=torch.bfloat16, device=self.dev)
                _chk(lib.rf_unet_upsample2(h, _ptr(cur), B_, H_, W_, C_, _ptr(y), s), "upsample2")
                tape.append(("up", cur.shape))
                cur = y
            elif step.startswith("skip") if isinstance(step, str) else False:
                skips[step] = cur
                last_skip = step
            elif isinstance(step, str) and step.startswith("cat:"):
                sk = skips[step[4:]]
                y = torch.empty((B_, H_, W_, C_ + sk.shape[3]), dtype=torch.bfloat16, device=self.dev)
                _chk(lib.rf_unet_concat(h, _ptr(cur), C_, _ptr(sk), sk.shape[3], B_ * H_ * W_, _ptr(y), 0, s), "cat")
                tape.append(("cat", C_, step[4:]))
                cur = y
            else:
                name, ci, co, relu = step
                y = torch.empty((B_, H_, W_, co), dtype=torch.bfloat16, device=self.dev)
                y32 = None
                if name == "out":
                    y32 = out32 = torch.empty((B_, H_, W_, co), dtype=torch.float32, device=self.dev)
                _chk(conv3x3(lib, h, _ptr(cur), B_, H_, W_, ci, _ptr(self.Wbf[name]), _ptr(self.b[name]), co,
                             int(relu), _ptr(y), _ptr(y32), s), "conv3x3")
                tape.append(("conv", name, cur, y, relu))
                cur = y
        self._tape = tape
        return out32

    # ---- backward -----------------------------------------------------------------
    def backward(self, dout):
        """dout: [B, H, W, cout] bfloat16 gradient of the loss wrt the output.
        Accumulates into the FP32 weight/bias gradients (call zero_grad
        first)."""
        lib, s, h = L.load(), _stream(), self.ctx.handle
        g = dout.contiguous()
        skip_grads = {}
        for rec in reversed(self._tape):
            kind = rec[0]
            if kind == "conv":
                _, name, xin, y, relu = rec
                B_, H_, W_, ci = xin.shape
                co = y.shape[3]
                if relu:
                    g = g.clone()
                    _chk(lib.rf_unet_relu_backward(h, _ptr(g), _ptr(y), g.numel(), s), "relu_bwd")
                _chk(conv3x3_wgrad(lib, h, _ptr(xin), _ptr(g), B_, H_, W_, ci, co, _ptr(self.gW[name]), s),
                     "wgrad")
                _chk(lib.rf_unet_bias_grad(h, _ptr(g), B_ * H_ * W_, co, _ptr(self.gb[name]), s), "bias_grad")
                if name == self.plan[0][0]:
                    g = None  # no gradient needed for the network input
                    continue
                dx = torch.empty((B_, H_, W_, ci), dtype=torch.bfloat16, device=self.dev)
                _chk(conv3x3(lib, h, _ptr(g), B_, H_, W_, co, _ptr(self.Wflip[name]), None, ci, 0, _ptr(dx), None,
                             s), "dgrad")
                g = dx
            elif kind == "cat":
                _, ca, sname = rec
                B_, H_, W_, C_ = g.shape
                main = torch.empty((B_, H_, W_, ca), dtype=torch.bfloat16, device=self.dev)
                skg = torch.empty((B_, H_, W_, C_ - ca), dtype=torch.bfloat16, device=self.dev)
                _chk(lib.rf_unet_concat(h, _ptr(main), ca, _ptr(skg), C_ - ca, B_ * H_ * W_, _ptr(g), 1, s), "split")
                skip_grads[sname] = skg
                g = main
            elif kind == "up":
                _, shp = rec
                dx = torch.empty(shp, dtype=torch.bfloat16, device=self.dev)
                _chk(lib.rf_unet_upsample2_backward(h, _ptr(g), shp[0], shp[1], shp[2], shp[3], _ptr(dx), s), "up_bwd")
                g = dx
            elif kind == "pool":
                _, shp, arg, sname = rec
                dx = torch.empty(shp, dtype=torch.bfloat16, device=self.dev)
                _chk(lib.rf_unet_maxpool2_backward(h, _ptr(g), _ptr(arg), shp[0], shp[1], shp[2], shp[3], _ptr(dx), s),
                     "pool_bwd")
                if sname in skip_grads:
                    _chk(lib.rf_unet_add(h, _ptr(dx), _ptr(skip_grads[sname]), dx.numel(), s), "add")
                g = dx
        self._tape = None

    def zero_grad(self):
        for k in self.gW:
            self.gW[k].zero_()
            self.gb[k].zero_()

    def mse(self, out32, target, mask=None):
        """Masked MSE of channel 0 vs target [B, H, W]; returns (loss tensor
        [1], dout bf16)."""
        lib, s = L.load(), _stream()
        B_, H_, W_, C_ = out32.shape
        npix = B_ * H_ * W_
        count = float(mask.sum().item()) if mask is not None else float(npix)
        loss = torch.zeros(1, dtype=torch.float32, device=self.dev)
        dout = torch.empty((B_, H_, W_, C_), dtype=torch.bfloat16, device=self.dev)
        # contiguous copies are bound to names: a temporary freed between two
        # argument evaluations could hand its memory to the next one
        target = target.contiguous()
        mask = mask.contiguous() if mask is not None else None
        _chk(lib.rf_unet_mse(self.ctx.handle, _ptr(out32), C_, _ptr(target), _ptr(mask), npix, count, _ptr(dout),
                             _ptr(loss), s), "mse")
        return loss, dout


def bench_conv(B=8, H=128, W=128, Cin=128, Cout=128, reps=20, tensor_cores=True):
    """Time one 3x3 convolution layer (BF16 NHWC, FP32 accumulation) with
    CUDA events: the tcgen05 kernel (tensor_cores=True) or the mma.sync one.
    Returns (ms per call, TFLOP/s)."""
    lib, s, ctx = L.load(), _stream(), Context.get(0)
    g = torch.Generator(device="cpu").manual_seed(0)
    x = torch.randn((B, H, W, Cin), generator=g).to(torch.bfloat16).cuda()
    w = (0.05 * torch.randn((Cout, 3, 3, Cin), generator=g)).to(torch.bfloat16).cuda()
    bias = torch.zeros(Cout, device="cuda")
    y = torch.empty((B, H, W, Cout), dtype=torch.bfloat16, device="cuda")
    fn = lib.rf_unet_conv3x3_tc if tensor_cores else lib.rf_unet_conv3x3
    call = lambda: _chk(fn(ctx.handle, _ptr(x), B, H, W, Cin, _ptr(w), _ptr(bias), Cout, 1, _ptr(y), None, s),
                        "conv3x3")
    for _ in range(3):
        call()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        call()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    return ms, 2.0 * B * H * W * Cout * 9 * Cin / (ms * 1e-3) / 1e12


def bench_wgrad(B, H, W, Cin, Cout, reps=20, tensor_cores=True):
    """Time the weight gradient of one 3x3 layer (rf_unet_conv3x3_wgrad_tc,
    or the mma.sync rf_unet_conv3x3_wgrad) on random data, the accumulator
    zeroed before each call.  Returns (ms per call, TFLOP/s)."""
    lib, s, ctx = L.load(), _stream(), Context.get(0)
    g = torch.Generator(device="cpu").manual_seed(0)
    x = torch.randn((B, H, W, Cin), generator=g).to(torch.bfloat16).cuda()
    dy = torch.randn((B, H, W, Cout), generator=g).to(torch.bfloat16).cuda()
    dw = torch.zeros((Cout, 3, 3, Cin), dtype=torch.float32, device="cuda")
    fn = lib.rf_unet_conv3x3_wgrad_tc if tensor_cores else lib.rf_unet_conv3x3_wgrad
    call = lambda: _chk(fn(ctx.handle, _ptr(x), _ptr(dy), B, H, W, Cin, Cout, _ptr(dw), s), "wgrad")
    for _ in range(3):
        call()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        call()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    return ms, 2.0 * B * H * W * Cout * 9 * Cin / (ms * 1e-3) / 1e12


if __name__ == "__main__":
    import argparse
    import json

    p = argparse.ArgumentParser(description="time one 3x3 convolution layer")
    p.add_argument("--shape", type=int, nargs=5, default=[8, 128, 128, 128, 128], metavar=("B", "H", "W", "CIN", "COUT"))
    p.add_argument("--reps", type=int, default=20)
    p.add_argument("--mma-sync", action="store_true", help="time the mma.sync kernel instead of tcgen05")
    p.add_argument("--wgrad", action="store_true", help="time the weight gradient instead of the convolution")
    a = p.parse_args()
    bench = bench_wgrad if a.wgrad else bench_conv
    ms, tf = bench(*a.shape, reps=a.reps, tensor_cores=not a.mma_sync)
    print(json.dumps({"shape": a.shape, "op": "wgrad" if a.wgrad else "conv",
                      "kernel": "mma.sync" if a.mma_sync else "tcgen05", "ms": ms, "tflops": tf}))
