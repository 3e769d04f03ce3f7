"""Autotuner for the forward solve's kernel variant and tile shape.

A shape is (band, block, variant, window): for the line-sweep variants a
sweep's lines are split into bands of `band` lines (one CTA each) advanced
`block` line steps per block; for the tile queue (variant 8) `band` is the
tile side (16 or 32) and `window` the delta-stepping window in tile
crossings (0 = the kernel's default).  The best shape depends on the grid
size and the GPU.  tune_sweep() times the candidate shapes on a real solve
and keeps the fastest per grid-size bucket (next power of two of
max(ny, nx)); results are cached in a JSON file keyed by the GPU name, so
later processes reuse them without timing again.  Cache entries without a
variant field (written before it existed) are ignored; entries without a
window read as window 0.

Cache file: $RF_AUTOTUNE_CACHE, else ~/.cache/rf_gb300/autotune.json.
"""
from __future__ import annotations

import json
import os
import threading

# (band, block, variant, window): 8 tile queue (band = tile side), 2 streamed, 1 tiled with one
# thread per node, 4 tiled with four
CANDIDATES = [(16, 0, 8, 0.0), (16, 0, 8, 2.0), (16, 0, 8, 8.0), (32, 0, 8, 0.0), (32, 0, 8, 4.0),
              (32, 32, 2, 0.0), (64, 16, 2, 0.0), (32, 16, 2, 0.0), (32, 32, 1, 0.0), (32, 32, 4, 0.0)]

_lock = threading.Lock()


def cache_path() -> str:
    p = os.environ.get("RF_AUTOTUNE_CACHE")
    if p:
        return p
    return os.path.join(os.path.expanduser("~"), ".cache", "rf_gb300", "autotune.json")


def bucket(ny: int, nx: int) -> int:
    """Next power of two of max(ny, nx)."""
    m = max(int(ny), int(nx), 1)
    b = 1
    while b < m:
        b *= 2
    return b


def _load() -> dict:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(d: dict) -> None:
    p = cache_path()
    os.makedirs(os.path.dirname(p), exist_ok=True)
    tmp = p + ".tmp"
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, p)


def lookup(device_name: str, ny: int, nx: int):
    """(band, block, variant, window) cached for this GPU and size bucket,
    or None."""
    with _lock:
        e = _load().get(device_name, {}).get(str(bucket(ny, nx)))
    if not e or "variant" not in e:
        return None
    return (int(e["band"]), int(e["block"]), int(e["variant"]), float(e.get("window", 0.0)))


def record(device_name: str, ny: int, nx: int, band: int, block: int, variant: int, window: float, ms: float,
           table=None) -> None:
    with _lock:
        d = _load()
        d.setdefault(device_name, {})[str(bucket(ny, nx))] = {"band": int(band), "block": int(block),
                                                              "variant": int(variant), "window": float(window),
                                                              "ms": float(ms), "timings": table or {}}
        _store(d)


def choose(timings: dict):
    """Fastest shape of {shape: ms}; ties go to the first."""
    best = None
    for shape, ms in timings.items():
        if best is None or ms < timings[best]:
            best = shape
    return best


def tune_sweep(proj5, eps, src, h, candidates=None, repeats=2, force=False):
    """Time rf_sweep_forward for each candidate (band, block, variant,
    window) on this input, cache and return the fastest.  Uses the cached
    result unless force."""
    import torch

    from . import api

    ny, nx = src.shape
    name = torch.cuda.get_device_name(proj5.device)
    if not force:
        hit = lookup(name, ny, nx)
        if hit is not None:
            return hit
    T = torch.empty((ny, nx), dtype=torch.float32, device=proj5.device)
    timings = {}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for band, block, variant, window in (candidates or CANDIDATES):
        o = api.make_opts(band=band, block=block, variant=variant, window=window)
        try:
            api.rf_sweep_forward(proj5, eps, src, h, opts=o, T=T, record=False)
        except Exception:
            continue  # shape not supported on this device
        torch.cuda.synchronize()
        e0.record()
        for _ in range(repeats):
            api.rf_sweep_forward(proj5, eps, src, h, opts=o, T=T, record=False)
        e1.record()
        torch.cuda.synchronize()
        timings[(band, block, variant, window)] = e0.elapsed_time(e1) / repeats
    api.Context.get(proj5.device).stats()
    best = choose(timings)
    record(name, ny, nx, *best, timings[best],
           {f"{b}x{k}x{n}x{w:g}": round(v, 4) for (b, k, n, w), v in timings.items()})
    return best


# batched solves: (band, variant, window) -- 8 the tile queue over all grids (band = tile side), 1 the
# persistent line-sweep kernel (whole grids per CTA)
BATCH_CANDIDATES = [(16, 8, 0.0), (16, 8, 2.0), (16, 8, 8.0), (32, 8, 0.0), (0, 1, 0.0)]


def batch_key(n_grids: int, total_nodes: int) -> str:
    return f"batch{int(n_grids)}x{bucket(int(total_nodes), 1)}"


def tune_batch(bs, candidates=None, repeats=2, force=False):
    """Time BatchSolver `bs` (api.BatchSolver, not yet captured) with each
    candidate (band, variant, window), cache and return the fastest; leaves
    bs.opts set to it.  Uses the cached result unless force."""
    import torch

    from . import api

    name = torch.cuda.get_device_name(bs.T.device)
    key = batch_key(bs.n, bs.total)
    if not force:
        with _lock:
            e = _load().get(name, {}).get(key)
        if e and "variant" in e:
            best = (int(e["band"]), int(e["variant"]), float(e.get("window", 0.0)))
            bs.opts = api.make_opts(band=best[0], variant=best[1], window=best[2])
            return best
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    timings = {}
    for cand in (candidates or BATCH_CANDIDATES):
        band, variant = cand[0], cand[1]
        window = cand[2] if len(cand) > 2 else 0.0
        bs.opts = api.make_opts(band=band, variant=variant, window=window)
        try:
            bs.run()
        except Exception:
            continue  # not supported for this batch (e.g. lines beyond the persistent kernel's limit)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(repeats):
            bs.run()
        e1.record()
        torch.cuda.synchronize()
        timings[(band, variant, window)] = e0.elapsed_time(e1) / repeats
    api.Context.get(bs.T.device).stats()
    best = choose(timings)
    bs.opts = api.make_opts(band=best[0], variant=best[1], window=best[2])
    with _lock:
        d = _load()
        d.setdefault(name, {})[key] = {"band": best[0], "variant": best[1], "window": best[2], "block": 0,
                                        "ms": timings[best],
                                        "timings": {f"{b}x{v}x{w:g}": round(t, 4) for (b, v, w), t in timings.items()}}
        _store(d)
    return best


def best_opts(device_name: str, ny: int, nx: int, **kw):
    """api.make_opts with the cached shape for this bucket (defaults otherwise)."""
    from . import api
    hit = lookup(device_name, ny, nx)
    if hit is not None:
        kw.setdefault("band", hit[0])
        kw.setdefault("block", hit[1])
        kw.setdefault("variant", hit[2])
        kw.setdefault("window", hit[3])
    return api.make_opts(**kw)
