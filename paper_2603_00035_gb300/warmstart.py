"""Learned warm start (a11, a12).

A 4-level U-Net (unet.UNet) maps (L, w, source mask, nearest-source
features) at 512 x 512 to an initial arrival-time field.  It is trained on
fields the solver itself generates (rf_batch_solve on synthetic inputs) with
the project's own forward/backward kernels.  For a large grid the fields are
box-averaged to 512^2, the network's guess is resampled bilinearly to the
grid, and the solve starts from it through rf_sweep_forward's replacement
update (RF_MODE_WARM), so an underestimate cannot freeze in.  Every warm
result is judged by the residual check (rf_residual); on failure or
non-convergence the solve is redone cold from +inf.
"""
from __future__ import annotations

import time

import numpy as np
import torch

from . import _lib as L
from . import api
from .api import Context, _ptr, _stream
from .unet import UNet

NET_RES = 512
N_PLANES = 9  # L11, L21, L22, wx, wy, source, distance, dx, dy
N_CH = 16


def source_list(src):
    """(src_ij int32 [nsrc, 2], src_off int32 [B+1]) of a uint8 [B, H, W] mask."""
    nz = torch.nonzero(src)
    b = nz[:, 0]
    counts = torch.bincount(b, minlength=src.shape[0])
    off = torch.zeros(src.shape[0] + 1, dtype=torch.int32, device=src.device)
    off[1:] = torch.cumsum(counts, 0).to(torch.int32)
    return nz[:, 1:].to(torch.int32).contiguous(), off


def features(proj, src, h, ctx=None):
    """Network input: proj [B, 5, H, W] projected fields, src [B, H, W] mask
    -> NHWC BF16 [B, H, W, 16]."""
    ctx = ctx or Context.get(proj.device)
    lib, s = L.load(), _stream()
    B, _, H, W = proj.shape
    planes = torch.empty((B, N_PLANES, H, W), dtype=torch.float32, device=proj.device)
    planes[:, :5] = proj
    planes[:, 5] = src.to(torch.float32)
    ij, off = source_list(src)
    feat = torch.empty((B, 3, H, W), dtype=torch.float32, device=proj.device)
    L.check(lib.rf_unet_source_features(ctx.handle, B, H, W, float(h), _ptr(ij), _ptr(off), _ptr(feat), s),
            "source_features")
    planes[:, 6:] = feat
    x = torch.empty((B, H, W, N_CH), dtype=torch.bfloat16, device=proj.device)
    L.check(lib.rf_unet_pack_input(ctx.handle, _ptr(planes), N_PLANES, B, H, W, N_CH, _ptr(x), s), "pack_input")
    return x


def batch_forward(proj, src, h, opts=None, ctx=None):
    """T [B, n, n] of B same-size grids (proj [B, 5, n, n] projected, src
    [B, n, n]) through one rf_batch_solve launch (forward + record only)."""
    ctx = ctx or Context.get(proj.device)
    B, _, n, m = proj.shape
    total = B * n * m
    packed = proj.permute(1, 0, 2, 3).contiguous()  # 5 planes of all grids
    desc = np.zeros(B, dtype=api._desc_dtype())
    for b in range(B):
        desc[b] = (n, m, h, 0, b * n * m)
    desc_t = torch.from_numpy(desc.view(np.uint8)).to(proj.device)
    T = torch.empty(total, dtype=torch.float32, device=proj.device)
    rec = api.Record(torch.empty(total, dtype=torch.uint8, device=proj.device),
                     torch.empty(total, dtype=torch.float32, device=proj.device),
                     torch.empty((5, total), dtype=torch.float32, device=proj.device))
    gstat = torch.zeros((B, 3), dtype=torch.int32, device=proj.device)
    o = opts if opts is not None else api.make_opts()
    import ctypes
    crec = rec.c()
    src_c = src.contiguous()
    L.check(L.load().rf_batch_solve(ctx.handle, _ptr(desc_t), B, total, max(n, m), _ptr(packed), 1e-6,
                                    _ptr(src_c), ctypes.byref(o), _ptr(T), ctypes.byref(crec), None, None,
                                    _ptr(gstat), _stream()), "rf_batch_solve")
    return T.view(B, n, m), gstat


def make_samples(seeds, n=NET_RES, eps=1e-6, delta=0.05, device="cuda"):
    """(x bf16 [B, n, n, 16], T [B, n, n]) for the given seeds: 8- or
    16-mode fields, |w| = 0.3, 1-8 sources, T from the solver."""
    from rf_inputs import gpu as G
    h = 1.0 / (n - 1)
    raws = []
    for s in seeds:
        K = 8 if s % 2 == 0 else 16
        raws.append(G.randers_fields_batch([s], n, h, K, eps, 0.3, device))
    raw = torch.cat(raws, 0)
    src, _ = G.random_sources_batch(seeds, n, 1, 8, device)
    B = raw.shape[0]
    flat = raw.permute(1, 0, 2, 3).contiguous().view(5, 1, B * n * n)
    proj_flat, _ = api.rf_project(flat, eps, delta)
    proj = proj_flat.view(5, B, n, n).permute(1, 0, 2, 3).contiguous()
    T, gstat = batch_forward(proj, src, h)
    return features(proj, src, h), T, gstat


def train(samples=10000, chunk=256, batch=8, lr=1e-3, seed=0, log=None, device="cuda"):
    """Train a UNet on `samples` solver-generated 512^2 samples (one pass)."""
    net = UNet(device=device, seed=seed)
    opt = torch.optim.Adam(net.parameters(), lr=lr)
    hist = []
    t0 = time.perf_counter()
    done = 0
    c = 0
    while done < samples:
        k = min(chunk, samples - done)
        seeds = list(range(seed * 1_000_000 + done, seed * 1_000_000 + done + k))
        x, T, gstat = make_samples(seeds, device=device)
        if int(gstat[:, 0].abs().sum()) != 0:
            raise RuntimeError("training-data solve failed")
        for b0 in range(0, k, batch):
            xb = x[b0:b0 + batch]
            out = net.forward(xb)
            loss, dout = net.mse(out, T[b0:b0 + batch].contiguous())
            net.zero_grad()
            net.backward(dout)
            net.attach_grads()
            opt.step()
            net.refresh()
            hist.append(float(loss))
        done += k
        c += 1
        if log:
            log(f"chunk {c}: samples {done}, loss {np.mean(hist[-max(1, k // batch):]):.3e}, "
                f"{time.perf_counter() - t0:.1f}s")
    return net, dict(loss_history=hist, seconds=time.perf_counter() - t0, samples=samples)


def guess(net, raw5, src, h, eps=1e-6, delta=0.05, res=NET_RES):
    """Initial T [N, N] for one N x N grid (N a multiple of res): fields
    box-averaged to res^2, network at res^2, node-aligned bilinear upsample."""
    ctx = net.ctx
    lib, s = L.load(), _stream()
    N = src.shape[0]
    f = N // res
    assert f * res == N and src.shape[1] == N
    proj, _ = api.rf_project(raw5, eps, delta)
    coarse = torch.empty((5, res, res), dtype=torch.float32, device=raw5.device)
    L.check(lib.rf_unet_box_down(ctx.handle, _ptr(proj), 5, N, N, f, _ptr(coarse), s), "box_down")
    ij = torch.nonzero(src)
    csrc = torch.zeros((1, res, res), dtype=torch.uint8, device=raw5.device)
    csrc[0, (ij[:, 0] // f).clamp(max=res - 1), (ij[:, 1] // f).clamp(max=res - 1)] = 1
    hres = h * (N - 1) / (res - 1)
    x = features(coarse[None], csrc, hres, ctx)
    out = net.forward(x)
    net._tape = None
    t_res = out[0, :, :, 0].contiguous()
    T0 = torch.empty((N, N), dtype=torch.float32, device=raw5.device)
    L.check(lib.rf_unet_bilinear(ctx.handle, _ptr(t_res), 1, res, res, N, N, 1.0, _ptr(T0), s), "bilinear")
    return proj, T0


def solve(net, raw5, src, h, eps=1e-6, delta=0.05, opts=None, residual_tol=None, inflate=1.1):
    """Warm-started forward solve with residual check and cold fallback.
    The guess is scaled by `inflate` before the sweeps: a replacement sweep
    lowers an overestimate as fast as a cold start fills +inf, while an
    underestimate only rises about one edge cost per sweep.  Returns
    (T, info)."""
    ctx = net.ctx
    t0 = time.perf_counter()
    proj, T = guess(net, raw5, src, h, eps, delta)
    if inflate != 1.0:
        T.mul_(inflate)
    o = opts if opts is not None else api.make_opts()
    ow = api.make_opts(tol=o.tol, max_sweeps=o.max_sweeps, warm=True, band=o.band, block=o.block, rtol=o.rtol,
                       variant=o.variant, window=o.window)
    api.rf_sweep_forward(proj, eps, src, h, opts=ow, T=T, record=False)
    st = ctx.stats()
    res = float(api.rf_residual(proj, eps, src, h, T).item())
    tmax = float(T[torch.isfinite(T)].max())
    tol = residual_tol if residual_tol is not None else 1e-5 * tmax
    info = dict(warm_sweeps=st["sweeps"], warm_status=st["status_name"], residual=res, fallback=False)
    if st["status"] != 0 or not st["converged"] or res > tol:
        api.rf_sweep_forward(proj, eps, src, h, opts=o, T=T, record=False)
        st2 = ctx.stats()
        info.update(fallback=True, cold_sweeps=st2["sweeps"], cold_status=st2["status_name"])
    torch.cuda.synchronize()
    info["seconds"] = time.perf_counter() - t0
    return T, info


def clear_underestimates(proj, src, h, T, eps=1e-6, ctx=None):
    """Set to +inf every node of the guess T whose value lies below the
    minimum of its valid candidates at T (residual < 0): such a value cannot
    be reached from its neighbours and would otherwise have to rise one edge
    cost per update.  Returns the number of nodes cleared."""
    mx, res = api.rf_residual(proj, eps, src, h, T, per_node=True, ctx=ctx)
    bad = (res < 0) & (src == 0)
    T.masked_fill_(bad, float("inf"))
    return int(bad.sum())


def compare(net, raw5, src, h, eps=1e-6, delta=0.05, inflate=1.1, loose=1e-4):
    """Cold and warm solves of one grid with the tile queue, timed with CUDA
    events: the exact solve (rtol 1e-6) cold from +inf, the same with a
    stopping tolerance of `loose`, and warm starts from the network's guess
    (inflated, and inflated with the underestimates cleared) at both
    tolerances; errors are max |T - T_cold exact| / max T.  The guess's own
    cost (network + resampling) is reported apart."""
    ctx = net.ctx
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    proj, _ = api.rf_project(raw5, eps, delta)

    def timed(fn):
        torch.cuda.synchronize()
        e0.record()
        out = fn()
        e1.record()
        torch.cuda.synchronize()
        return out, e0.elapsed_time(e1)

    def solve(T, rtol, warm):
        o = api.make_opts(rtol=rtol, warm=warm, max_sweeps=1000)
        api.rf_sweep_forward(proj, eps, src, h, opts=o, T=T, record=False)
        return T

    T_ref = torch.empty(src.shape, dtype=torch.float32, device=raw5.device)
    solve(T_ref, 1e-6, False)  # warm-up of the workspace
    _, ms_cold = timed(lambda: solve(T_ref, 1e-6, False))
    st_cold = ctx.stats()
    tmax = float(T_ref[torch.isfinite(T_ref)].max())
    rows = {"cold_exact": dict(ms=ms_cold, rounds=st_cold["rounds"], updates_per_node=st_cold["cell_updates"] / src.numel(),
                               err=0.0, status=st_cold["status_name"])}

    def err(T):
        d = (T - T_ref).abs()
        d = torch.where(torch.isfinite(T_ref), d, torch.zeros_like(d))
        return float(d.max()) / tmax

    T = torch.empty_like(T_ref)
    _, ms = timed(lambda: solve(T, loose, False))
    st = ctx.stats()
    rows["cold_loose"] = dict(ms=ms, rounds=st["rounds"], updates_per_node=st["cell_updates"] / src.numel(),
                              err=err(T), status=st["status_name"])
    (_, T0), ms_guess = timed(lambda: guess(net, raw5, src, h, eps, delta))
    rows["guess"] = dict(ms=ms_guess, err=err(T0 * inflate))
    for clear in (False, True):
        for rtol, tag in ((1e-6, "exact"), (loose, "loose")):
            T = (T0 * inflate).contiguous()
            n_clear = 0

            def run():
                nonlocal n_clear
                if clear:
                    n_clear = clear_underestimates(proj, src, h, T, eps, ctx)
                return solve(T, rtol, True)
            _, ms = timed(run)
            st = ctx.stats()
            rows[f"warm{'_cleared' if clear else ''}_{tag}"] = dict(
                ms=ms, rounds=st["rounds"], updates_per_node=st["cell_updates"] / src.numel(), err=err(T),
                status=st["status_name"], cleared=n_clear)
    return rows


def main():
    import argparse
    import json

    p = argparse.ArgumentParser(description="train the warm-start network, then cold vs warm solves")
    p.add_argument("--samples", type=int, default=10000)
    p.add_argument("--eval-n", type=int, default=4096)
    p.add_argument("--eval-grids", type=int, default=3)
    p.add_argument("--save", default="")
    a = p.parse_args()
    import sys
    import os
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import rf_inputs as R

    net, tr = train(samples=a.samples, log=lambda m: print(m, file=sys.stderr, flush=True))
    if a.save:
        torch.save(net.state_dict(), a.save)
    n = a.eval_n
    h = 1.0 / (n - 1)
    evals = []
    for k in range(a.eval_grids):
        raw = torch.from_numpy(R.randers_fields(n, n, h, 16, 900 + k, omega="unit", omega_scale=0.3)).cuda()
        src = torch.from_numpy(R.random_sources(n, n, 1 + (k % 8), 900 + k)).cuda()
        evals.append(dict(grid=n, sources=int(src.sum()), **compare(net, raw, src, h)))
        print(json.dumps(evals[-1]), file=sys.stderr, flush=True)
    print(json.dumps(dict(train=dict(samples=tr["samples"], seconds=tr["seconds"],
                                     loss_first=tr["loss_history"][0], loss_last=float(np.mean(tr["loss_history"][-20:]))),
                          eval=evals)))


if __name__ == "__main__":
    main()
