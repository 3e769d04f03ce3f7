"""Covariate -> metric encoder trained end to end through the solver (Sec. 5,
"Encoder Architecture"; the synthetic covariates of App. "Synthetic
Propagation Scenarios" stand in for the wildfire data).

Two pathways, both on librf's BF16 convolution kernels:
* global: the domain-wide covariates y (wind, temperature) pass through an
  MLP giving the baseline (G0, b0); the MLP's dense layers run as 3x3
  convolutions on a 1x1 image (only the centre tap sees data);
* spatial: the covariate planes Y(x) (terrain, fuel) pass through a
  fully-convolutional U-Net giving per-node residuals (G_local, b_local).
The head combines them as G = G0 + alpha G_local, b = b0 + alpha b_local
(rf_encoder_combine); the App. B projection makes them feasible; the solve
and its adjoint give dL/dT -> dL/d(G, b) (Alg. 2); the head's adjoint and
the networks' backward passes carry it to the weights.  Every step runs in
librf's kernels; torch holds the tensors and the Adam update.
"""
from __future__ import annotations

import time

import numpy as np
import torch

from . import _lib as L
from . import api
from .api import Context, _ptr, _stream
from .autograd import TotalVariation, metric_solve
from .unet import UNet

N_CH = 16  # network channels of the inputs and outputs


def mlp_plan(cin=N_CH, width=32, cout=N_CH):
    return [("m0", cin, width, True), ("m1", width, width, True), ("out", width, cout, False)]


class Encoder:
    def __init__(self, base=16, alpha=0.5, seed=0, device="cuda", g0=1.5):
        self.dev = torch.device(device)
        self.ctx = Context.get(self.dev)
        self.alpha = float(alpha)
        self.fcn = UNet(cin=N_CH, base=base, cout=N_CH, device=device, seed=seed, ctx=self.ctx)
        self.mlp = UNet(device=device, seed=seed + 1, ctx=self.ctx, plan=mlp_plan())
        # start from an isotropic metric g0 I and no drift (inside the
        # projection's bounds, so the clamp passes gradients)
        self.mlp.b["out"][0] = g0
        self.mlp.b["out"][2] = g0
        self._shape = None

    def parameters(self):
        return self.fcn.parameters() + self.mlp.parameters()

    def forward(self, Y, y):
        """Y: [B, H, W, 16] BF16 spatial covariates, y: [B, 1, 1, 16] BF16
        global covariates -> gb [B, 5, H, W] FP32 (raw G, b per grid)."""
        B, H, W, _ = Y.shape
        local = self.fcn.forward(Y)
        base = self.mlp.forward(y)
        gb = torch.empty((B, 5, H, W), dtype=torch.float32, device=self.dev)
        L.check(L.load().rf_encoder_combine(self.ctx.handle, _ptr(local), B, H, W, N_CH, _ptr(base), N_CH,
                                            self.alpha, _ptr(gb), _stream()), "rf_encoder_combine")
        self._shape = (B, H, W)
        return gb

    def backward(self, dgb):
        B, H, W = self._shape
        dlocal = torch.empty((B, H, W, N_CH), dtype=torch.bfloat16, device=self.dev)
        dbase = torch.empty((B, 1, 1, N_CH), dtype=torch.bfloat16, device=self.dev)
        dgb = dgb.contiguous()  # held for the call (a temporary's memory could be reused)
        L.check(L.load().rf_encoder_combine_backward(self.ctx.handle, _ptr(dgb), B, H, W, N_CH, N_CH,
                                                     self.alpha, _ptr(dlocal), _ptr(dbase), _stream()),
                "rf_encoder_combine_backward")
        self.fcn.backward(dlocal)
        self.mlp.backward(dbase)

    def zero_grad(self):
        self.fcn.zero_grad()
        self.mlp.zero_grad()

    def attach_grads(self):
        self.fcn.attach_grads()
        self.mlp.attach_grads()

    def refresh(self):
        self.fcn.refresh()
        self.mlp.refresh()


def pack(samples, device):
    """Covariate samples (rf_inputs.covariate_sample) -> BF16 network inputs,
    true fields, grid spacing."""
    Y = np.stack([s["Y"] for s in samples])
    B, H, W, c = Y.shape
    Yp = np.zeros((B, H, W, N_CH), np.float32)
    Yp[..., :c] = Y
    yp = np.zeros((B, 1, 1, N_CH), np.float32)
    yp[:, 0, 0, :3] = np.stack([s["y"] for s in samples])
    gb = np.stack([s["gb"] for s in samples])
    t = lambda a: torch.from_numpy(a).to(device)
    return t(Yp).to(torch.bfloat16), t(yp).to(torch.bfloat16), t(gb), samples[0]["h"]


def observations(gb_true, sources, obs, h, prm):
    """Observed arrival times: the solve of the true fields from each source
    mask, kept at the observed nodes."""
    out = []
    with torch.no_grad():
        for b in range(gb_true.shape[0]):
            _, proj = api.rf_metric_project(gb_true[b].contiguous(), prm, want_gbp=False)
            row = []
            for s, o in zip(sources[b], obs[b]):
                T, _ = api.rf_sweep_forward(proj, prm.eps, s, h, record=False)
                row.append(torch.where(o.bool(), T, torch.zeros_like(T)))
            out.append(row)
    return out


def data_loss(enc, Y, y, sources, obs, targets, h, prm, tv_weight=0.0):
    """Mean over grids of 1/2 sum_obs (T - T^)^2 / |obs| (+ TV), with the
    gradient wrt the raw encoder output."""
    gb = enc.forward(Y, y).requires_grad_(True)
    B = gb.shape[0]
    loss = torch.zeros((), device=gb.device)
    for b in range(B):
        for s, o, tgt in zip(sources[b], obs[b], targets[b]):
            T, gbp = metric_solve(gb[b], s, h, prm)
            d = torch.where(o.bool(), T - tgt, torch.zeros_like(T))
            loss = loss + 0.5 * (d * d).sum() / (o.sum() * B)
        if tv_weight > 0:
            loss = loss + TotalVariation.apply(gbp, "frobenius", tv_weight / B, tv_weight / B)
    return loss, gb


def train_synthetic(steps=300, batch=8, n=64, n_sources=2, obs_frac=0.1, lr=2e-3, seed=0, eval_batches=2,
                    tv_weight=0.0, log_every=50, device="cuda", alpha=0.5):
    """Train the encoder on fresh synthetic samples every step; report the
    held-out recovery of G and b and of the arrival times, against the
    untrained encoder and a constant-metric baseline."""
    import rf_inputs as R

    dev = torch.device(device)
    prm = api.metric_params(0.3, 5.0, None, 0.05, 1e-6)
    enc = Encoder(seed=seed, device=device, alpha=alpha)
    opt = torch.optim.Adam(enc.parameters(), lr=lr)

    def batch_of(k):
        samples = [R.covariate_sample(n, 100000 * seed + k * batch + i) for i in range(batch)]
        Y, y, gb_true, h = pack(samples, dev)
        sources = [[torch.from_numpy(R.random_sources(n, n, 1, 7919 * (k * batch + i) + j, margin=4)).to(dev)
                    for j in range(n_sources)] for i in range(batch)]
        obs = [[torch.from_numpy(R.observation_mask(n, n, obs_frac, 104729 * (k * batch + i) + j)).to(dev)
                for j in range(n_sources)] for i in range(batch)]
        return Y, y, gb_true, h, sources, obs

    held = [batch_of(10 ** 6 + k) for k in range(eval_batches)]

    def evaluate():
        errs = {"g": [], "b": [], "T": []}
        with torch.no_grad():
            for Y, y, gb_true, h, sources, obs in held:
                gb = enc.forward(Y, y)
                for b in range(gb.shape[0]):
                    gbp, proj = api.rf_metric_project(gb[b].contiguous(), prm)
                    gt = gb_true[b]
                    errs["g"].append(float(torch.linalg.vector_norm(gbp[:3] - gt[:3]) /
                                           torch.linalg.vector_norm(gt[:3])))
                    nb = torch.linalg.vector_norm(gt[3:])
                    errs["b"].append(float(torch.linalg.vector_norm(gbp[3:] - gt[3:]) / max(float(nb), 1e-6)))
                    _, projt = api.rf_metric_project(gt.contiguous(), prm, want_gbp=False)
                    for s in sources[b]:
                        T, _ = api.rf_sweep_forward(proj, prm.eps, s, h, record=False)
                        Tt, _ = api.rf_sweep_forward(projt, prm.eps, s, h, record=False)
                        errs["T"].append(float(torch.linalg.vector_norm(T - Tt) / torch.linalg.vector_norm(Tt)))
        return {k: float(np.mean(v)) for k, v in errs.items()}

    def constant_baseline():
        # a constant isotropic metric at the mean of the true g; its arrival
        # times are taken with the TRUE drift (an upper bound on what the
        # spatial pathway must add)
        errs = {"g": [], "b": [], "T_with_true_b": []}
        with torch.no_grad():
            for _, _, gb_true, h, sources, _ in held:
                gbar = float(gb_true[:, 0].mean())
                for b in range(gb_true.shape[0]):
                    gt = gb_true[b]
                    c = gt.clone()
                    c[0] = c[2] = gbar
                    c[1] = 0.0
                    errs["g"].append(float(torch.linalg.vector_norm(c[:3] - gt[:3]) /
                                           torch.linalg.vector_norm(gt[:3])))
                    errs["b"].append(1.0)
                    _, projc = api.rf_metric_project(c.contiguous(), prm, want_gbp=False)
                    _, projt = api.rf_metric_project(gt.contiguous(), prm, want_gbp=False)
                    for s in sources[b]:
                        T, _ = api.rf_sweep_forward(projc, prm.eps, s, h, record=False)
                        Tt, _ = api.rf_sweep_forward(projt, prm.eps, s, h, record=False)
                        errs["T_with_true_b"].append(float(torch.linalg.vector_norm(T - Tt) /
                                                           torch.linalg.vector_norm(Tt)))
        return {k: float(np.mean(v)) for k, v in errs.items()}

    before = evaluate()
    hist = []
    t0 = time.perf_counter()
    for k in range(steps):
        Y, y, gb_true, h, sources, obs = batch_of(k)
        targets = observations(gb_true, sources, obs, h, prm)
        opt.zero_grad(set_to_none=True)
        enc.zero_grad()
        loss, gb = data_loss(enc, Y, y, sources, obs, targets, h, prm, tv_weight)
        loss.backward()
        enc.backward(gb.grad)
        enc.attach_grads()
        opt.step()
        enc.refresh()
        if log_every and (k % log_every == 0 or k == steps - 1):
            hist.append((k, float(loss.detach())))
    torch.cuda.synchronize()
    seconds = time.perf_counter() - t0
    after = evaluate()
    st = Context.get(dev).stats()
    return dict(steps=steps, batch=batch, n=n, sources=n_sources, observed_fraction=obs_frac, loss_history=hist,
                held_out_before=before, held_out_after=after, constant_metric_baseline=constant_baseline(),
                seconds=seconds, ms_per_step=1e3 * seconds / steps, status=st["status"])


def main():
    import argparse
    import json
    import os
    import sys

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    p = argparse.ArgumentParser(description="train the covariate encoder through the solver")
    p.add_argument("--steps", type=int, default=300)
    p.add_argument("--batch", type=int, default=8)
    p.add_argument("--n", type=int, default=64)
    p.add_argument("--seed", type=int, default=0)
    p.add_argument("--sources", type=int, default=2)
    p.add_argument("--obs", type=float, default=0.1)
    p.add_argument("--lr", type=float, default=2e-3)
    p.add_argument("--alpha", type=float, default=0.5)
    p.add_argument("--tv", type=float, default=0.0)
    a = p.parse_args()
    print(json.dumps(train_synthetic(steps=a.steps, batch=a.batch, n=a.n, n_sources=a.sources, obs_frac=a.obs,
                                     seed=a.seed, lr=a.lr, alpha=a.alpha, tv_weight=a.tv)))


if __name__ == "__main__":
    main()
