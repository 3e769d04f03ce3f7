"""Inverse metric problem (Sec. 4, Eq. 8) driven through the solver.

run_inverse: the factor-form parameterisation,

    min_theta  1/2 sum_{i in obs} (T_i(theta) - T_hat_i)^2

over theta = (L11, L21, L22, wx, wy) on every node, with Adam at the
paper's step sizes (1e-2 for the metric, 5e-3 for the drift; Sec. 4).  The
projection inside RFSolve keeps M SPD and the drift feasible.  The
observations come from a ground-truth solve of a known field; the initial
guess is M = I, w = 0 (the paper does not state one).

run_inverse_paper / paper_experiments: the paper's own parameterisation
(G, b) with the App. B projections and TV regularisers, and its 80 x 80
synthetic recoveries (isotropic, drift, multi-source, TV ablation).
"""
from __future__ import annotations

import time

import torch

from . import api
from .autograd import TotalVariation, metric_solve, rf_solve


def metric_from_raw(raw5, eps):
    l11, l21, l22 = raw5[0], raw5[1], raw5[2]
    return torch.stack([l11 * l11 + eps, l11 * l21, l21 * l21 + l22 * l22 + eps])


def run_inverse(raw_true, src, obs, h, steps=200, eps=1e-6, delta=0.05, lr_metric=1e-2, lr_drift=5e-3,
                algo="tiles", log_every=0):
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


def run_inverse_paper(gb_true, sources, obs, h, mode="iso", steps=300, init=1.5, tv_weight=1e-3,
                      tv_metric="frobenius", prm=None, lr_metric=1e-2, lr_drift=5e-3, clip=1.0, algo="tiles",
                      opts=None, noise=0.0, seed=0):
    """The paper's synthetic inverse experiments (Eq. 8; App. "Inverse
    Problem Experiments") in its own parameterisation (G, b):

        min 1/2 sum_s sum_{i in obs_s} (T_i^s - T^_i^s)^2 + w (R(G) + R(b))

    with T^s the solve of source mask s on the true fields.  Each iteration
    evaluates the data term through the App. B projection, the solves and
    the stencil-record adjoint, adds the TV gradient, takes an Adam step
    (learning rates 1e-2 for G and 5e-3 for b, gradient norm clipped, cosine
    decay) and projects the parameters back onto the feasible set (projected
    gradient descent).

    mode "iso": G = g I with g free (b fixed to the truth); "drift": b free
    per node (G fixed to the truth); "drift_const": one constant drift
    vector b free (G fixed to the truth; the appendix's constant-drift
    example read as a two-parameter problem); "full": all five fields free.  gb_true: float32
    CUDA (5, ny, nx); sources: list of uint8 (ny, nx) masks; obs: list of
    uint8 masks (one per source); noise: Gaussian noise added to the observed
    times, as a fraction of their standard deviation.  Returns the loss
    history, relative errors (of the fields, and of the drift's mean) and
    timing."""
    dev = gb_true.device
    prm = prm or api.metric_params()
    ny, nx = gb_true.shape[1:]
    with torch.no_grad():
        _, proj_true = api.rf_metric_project(gb_true, prm, want_gbp=False)
        targets = [api.rf_sweep_forward(proj_true, prm.eps, s, h, record=False)[0] for s in sources]
    obs_f = [o.to(torch.float32) for o in obs]
    if noise > 0:
        gen = torch.Generator(device="cpu").manual_seed(int(seed))
        targets = [t + noise * float(t[o.bool()].std()) * torch.randn(t.shape, generator=gen).to(dev)
                   for o, t in zip(obs, targets)]
    targets = [torch.where(o.bool(), t, torch.zeros_like(t)) for o, t in zip(obs, targets)]
    z = torch.zeros((ny, nx), dtype=torch.float32, device=dev)
    if mode == "iso":
        params = [torch.nn.Parameter(torch.full((ny, nx), float(init), device=dev))]
        groups = [{"params": params, "lr": lr_metric}]
        assemble = lambda: torch.stack([params[0], z, params[0], gb_true[3], gb_true[4]])
    elif mode == "drift":
        params = [torch.nn.Parameter(torch.full((2, ny, nx), float(init), device=dev))]
        groups = [{"params": params, "lr": lr_drift}]
        assemble = lambda: torch.cat([gb_true[:3], params[0]])
    elif mode == "drift_const":
        params = [torch.nn.Parameter(torch.full((2,), float(init), device=dev))]
        groups = [{"params": params, "lr": lr_drift}]
        assemble = lambda: torch.cat([gb_true[:3], params[0].view(2, 1, 1).expand(2, ny, nx)])
    elif mode == "full":
        g0 = torch.stack([torch.full((ny, nx), float(init), device=dev), z, torch.full((ny, nx), float(init),
                                                                                    device=dev)])
        params = [torch.nn.Parameter(g0), torch.nn.Parameter(torch.zeros((2, ny, nx), device=dev))]
        groups = [{"params": [params[0]], "lr": lr_metric}, {"params": [params[1]], "lr": lr_drift}]
        assemble = lambda: torch.cat([params[0], params[1]])
    else:
        raise ValueError(mode)
    opt = torch.optim.Adam(groups)
    sched = torch.optim.lr_scheduler.CosineAnnealingLR(opt, steps, eta_min=0.1 * lr_drift)
    hist = []
    t0 = time.perf_counter()
    for it in range(steps):
        opt.zero_grad(set_to_none=True)
        gb = assemble()
        loss = torch.zeros((), device=dev)
        gbp = None
        for s, o, tgt in zip(sources, obs_f, targets):
            T, gbp = metric_solve(gb, s, h, prm, algo, opts)
            d = torch.where(o.bool(), T - tgt, torch.zeros_like(T))
            loss = loss + 0.5 * (d * d * o).sum()
        if tv_weight > 0:
            loss = loss + TotalVariation.apply(gbp, tv_metric, tv_weight, tv_weight)
        loss.backward()
        if clip:
            torch.nn.utils.clip_grad_norm_(params, clip)
        opt.step()
        sched.step()
        with torch.no_grad():  # projection onto the feasible set
            gbp_new, _ = api.rf_metric_project(assemble().contiguous(), prm, want_proj=False)
            if mode == "iso":
                params[0].copy_(gbp_new[0])
            elif mode == "drift":
                params[0].copy_(gbp_new[3:])
            elif mode == "drift_const":
                params[0].copy_(gbp_new[3:].mean(dim=(1, 2)))
            else:
                params[0].copy_(gbp_new[:3])
                params[1].copy_(gbp_new[3:])
        if it % 10 == 0 or it == steps - 1:
            hist.append((it, float(loss.detach())))
    torch.cuda.synchronize()
    elapsed = time.perf_counter() - t0
    with torch.no_grad():
        gb = assemble()
        rel = lambda a, b: float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))
        out = dict(mode=mode, steps=steps, sources=len(sources), observations=int(sum(int(o.sum()) for o in obs)),
                   tv_weight=tv_weight, final_loss=hist[-1][1], loss_history=hist, seconds=elapsed,
                   ms_per_iteration=1e3 * elapsed / steps)
        if mode in ("iso", "full"):
            out["rel_err_metric"] = rel(gb[:3], gb_true[:3])
        if mode in ("drift", "drift_const", "full"):
            out["rel_err_b1"] = rel(gb[3], gb_true[3])
            out["rel_err_b2"] = rel(gb[4], gb_true[4])
            for c in (3, 4):
                m_true = float(gb_true[c].mean())
                out[f"rel_err_b{c - 2}_mean"] = abs(float(gb[c].mean()) - m_true) / abs(m_true)
    return out


def paper_experiments(steps=300, seed=0, device="cuda"):
    """The synthetic recoveries of the paper's inverse-problem section on an
    80 x 80 grid (h = 1/79): isotropic piecewise metric (g = 1 | 2) with
    full and 7 % observations, constant drift (0.15, 0.08) under G = I,
    multi-source recovery with 1, 2, 3, 5 sources at 7 % each, and the TV
    weight ablation on full observations with 2 % noise.  Yields one result
    dict per run."""
    import numpy as np

    import rf_inputs as R

    n, h = 80, 1.0 / 79
    dev = torch.device(device)
    t = lambda a: torch.from_numpy(a).to(dev)
    iso = t(R.piecewise_isotropic(n))
    centre = [t(R.point_sources(n, n, [(n // 2, n // 2)]))]
    full = [t(np.ones((n, n), np.uint8))]
    sparse = lambda k: [t(R.observation_mask(n, n, 0.07, seed + 17 * i)) for i in range(k)]
    yield dict(run="isotropic_full_obs", **run_inverse_paper(iso, centre, full, h, "iso", steps))
    yield dict(run="isotropic_7pct_obs", **run_inverse_paper(iso, centre, sparse(1), h, "iso", steps))
    drift = t(R.constant_gb(n, (1.0, 0.0, 1.0), (0.15, 0.08)))
    for w in (1e-3, 1e-2, 1e-1):
        yield dict(run=f"drift_full_obs_tv{w:g}", **run_inverse_paper(drift, centre, full, h, "drift", steps, init=0.0,
                                                                     tv_weight=w))
    yield dict(run="drift_constant_full_obs", **run_inverse_paper(drift, centre, full, h, "drift_const", steps,
                                                                  init=0.0, tv_weight=0.0))
    for k in (1, 2, 3, 5):
        srcs = [t(m) for m in (R.random_sources(n, n, 1, seed + 101 * i, margin=8) for i in range(k))]
        yield dict(run=f"multisource_{k}", **run_inverse_paper(iso, srcs, sparse(k), h, "iso", steps))
    for w in (0.0, 1e-4, 1e-3, 1e-2, 1e-1):
        yield dict(run=f"tv_ablation_{w:g}", **run_inverse_paper(iso, centre, full, h, "iso", steps, tv_weight=w,
                                                                 noise=0.02, seed=seed))


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
    p.add_argument("--algo", default="tiles")
    p.add_argument("--paper", action="store_true",
                   help="run the paper's 80x80 synthetic recoveries in its (G, b) parameterisation")
    a = p.parse_args()
    if a.paper:
        for r in paper_experiments(steps=a.steps if a.steps != 200 else 300, seed=a.seed):
            r.pop("loss_history")
            print(json.dumps(r), flush=True)
        return
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
