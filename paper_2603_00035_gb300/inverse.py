"""Inverse metric problem (Sec. 4, Eq. 8) driven through RFSolve.

    min_theta  1/2 sum_{i in obs} (T_i(theta) - T_hat_i)^2

over theta = (L11, L21, L22, wx, wy) on every node, with Adam at the
paper's step sizes (1e-2 for the metric, 5e-3 for the drift; Sec. 4).  The
projection inside RFSolve keeps M SPD and the drift feasible.  The TV
regularisers of Eq. 8 are not part of this driver.

The observations come from a ground-truth solve of a known field; the
initial guess is M = I, w = 0 (the paper does not state one).  Returns the
loss history and the relative recovery error of M and w.
"""
from __future__ import annotations

import time

import torch

from . import api
from .autograd import rf_solve


def metric_from_raw(raw5, eps):
    l11, l21, l22 = raw5[0], raw5[1], raw5[2]
    return torch.stack([l11 * l11 + eps, l11 * l21, l21 * l21 + l22 * l22 + eps])


def run_inverse(raw_true, src, obs, h, steps=200, eps=1e-6, delta=0.05, lr_metric=1e-2, lr_drift=5e-3,
                algo="ordered", log_every=0):
    """raw_true: (5, ny, nx) float32 CUDA ground truth; src, obs: uint8 masks."""
    dev = raw_true.device
    with torch.no_grad():
        proj_true, _ = api.rf_project(raw_true, eps, delta)
        T_true, _ = api.rf_sweep_forward(proj_true, eps, src, h, record=False)
    obs_f = obs.to(torch.float32)
    target = torch.where(obs.bool(), T_true, torch.zeros_like(T_true))
    ny, nx = src.shape
    init = torch.zeros((5, ny, nx), dtype=torch.float32, device=dev)
    init[0] = 1.0
    init[2] = 1.0
    L = torch.nn.Parameter(init[:3].clone())
    W = torch.nn.Parameter(init[3:].clone())
    opt = torch.optim.Adam([{"params": [L], "lr": lr_metric}, {"params": [W], "lr": lr_drift}])
    hist = []
    t0 = time.perf_counter()
    for it in range(steps):
        opt.zero_grad(set_to_none=True)
        raw = torch.cat([L, W], dim=0)
        T = rf_solve(raw, src, h, eps, delta, algo)
        diff = torch.where(obs.bool(), T - target, torch.zeros_like(T))
        loss = 0.5 * (diff * diff * obs_f).sum()
        loss.backward()
        opt.step()
        if log_every and (it % log_every == 0 or it == steps - 1):
            hist.append((it, float(loss.detach())))
    torch.cuda.synchronize()
    elapsed = time.perf_counter() - t0
    with torch.no_grad():
        raw = torch.cat([L, W], dim=0)
        m_est = metric_from_raw(raw, eps)
        m_true = metric_from_raw(raw_true, eps)
        proj_est, _ = api.rf_project(raw.contiguous(), eps, delta)
        rel_m = float(torch.linalg.vector_norm(m_est - m_true) / torch.linalg.vector_norm(m_true))
        rel_w = float(torch.linalg.vector_norm(proj_est[3:] - proj_true[3:]) /
                      torch.linalg.vector_norm(proj_true[3:]))
        T_fin = rf_solve(raw, src, h, eps, delta, algo)
        final = 0.5 * float((torch.where(obs.bool(), T_fin - target, torch.zeros_like(T_fin)) ** 2).sum())
    return dict(loss_history=hist, final_loss=final, rel_err_metric=rel_m, rel_err_drift=rel_w,
                seconds=elapsed, steps=steps)


def main():
    import argparse
    import json
    import os
    import sys

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import rf_inputs as R

    p = argparse.ArgumentParser(description="inverse metric problem on synthetic fields")
    p.add_argument("--n", type=int, default=2048)
    p.add_argument("--steps", type=int, default=200)
    p.add_argument("--obs", type=float, default=0.005)
    p.add_argument("--seed", type=int, default=0)
    p.add_argument("--algo", default="ordered")
    a = p.parse_args()
    c = R.config_inverse(n=a.n, seed=a.seed)
    dev = torch.device("cuda")
    raw_true = torch.from_numpy(c["raw"]).to(dev)
    src = torch.from_numpy(c["src"]).to(dev)
    obs = torch.from_numpy(R.observation_mask(a.n, a.n, a.obs, a.seed)).to(dev)
    out = run_inverse(raw_true, src, obs, c["h"], steps=a.steps, algo=a.algo, log_every=max(1, a.steps // 10))
    out["n"] = a.n
    out["observed_fraction"] = a.obs
    out["ms_per_step"] = 1e3 * out["seconds"] / a.steps
    print(json.dumps(out))


if __name__ == "__main__":
    main()
