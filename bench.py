"""Benchmark: forward+adjoint solves/s of the differentiable Randers eikonal
solver on a 2048x2048 grid (the inverse-problem workload), one GB300.

A step is one pass of the whole hot path over one grid: feasibility
projection -> forward fast sweep -> stencil record -> adjoint (lambda and
parameter gradients) -> projection backward, on seeded synthetic fields
(16-mode Fourier metric, |w| = 0.3 drift, 4 sources, dL/dT on 0.5 % of the
nodes).  Inputs are resident in HBM when the timed region starts; L2 is
flushed (a 256 MB write) between timed steps.  `e2e` repeats the step
through the public API from pinned HOST buffers with the host<->device
copies inside the timed region.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
With N > 1 (torchrun), every rank solves its own grid (independent
replicas; a single grid does not shard) and the value is the whole-job
aggregate.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "forward+adjoint solves/s at 2048x2048"
UNIT = "solves/s"
ALG_BYTES_PER_UPDATE = 28  # 5 fields x 4 B + T read 4 B + T write 4 B per node-update
# DRAM bytes (read + write) of one launch of the tile-queue forward kernel on the 2048^2 workload (16x16
# tiles), by delta-stepping window, each from one ncu capture (dram__bytes_read.sum + dram__bytes_write.sum).
# Reported as roofline.traffic only while the kernel's sources hash to the captured build's.
TRAFFIC_CAPTURES = {("tile_solve_kernel<16>", 2048, 2.0): {"sources_sha16": "ec162a0fb8fa3692", "bytes": 423551232 + 43747328},
                    ("tile_solve_kernel<16>", 2048, 4.0): {"sources_sha16": "ec162a0fb8fa3692", "bytes": 427654656 + 46024448}}
TRAFFIC_SOURCES = ["paper_2603_00035_gb300/csrc/rf_sweep_tiles.cu", "paper_2603_00035_gb300/csrc/rf_cone.cuh",
                   "paper_2603_00035_gb300/csrc/rf_sweep_common.cuh", "paper_2603_00035_gb300/csrc/rf_device.cuh"]
# kernels of ours per step: project, record, project backward; the forward variant's kernels (init and
# source check, then tile queue: plan, reset, seed, finish-seed, solve, stats; streamed: node records +
# sweep; tiled: sweep); the adjoint's (sweep: 1; ordered: epoch, keys, gather, unreached; levels: epoch,
# keys, depth, starts, gather, unreached; tiles: epoch, tile keys, tile gather -- CUB's sort kernels not
# counted)
LAUNCHES_BASE = 3
LAUNCHES_FORWARD = {8: 8, 2: 4, 1: 3, 4: 3}
LAUNCHES_ADJOINT = {"sweep": 1, "ordered": 4, "levels": 6, "tiles": 3}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--size", type=int, default=2048)
    p.add_argument("--algo", default="tiles", choices=["sweep", "ordered", "levels", "tiles"])
    p.add_argument("--band", type=int, default=0)
    p.add_argument("--block", type=int, default=0)
    p.add_argument("--variant", type=int, default=0, choices=[0, 1, 2, 4, 8],
                   help="forward kernel (0: autotuned; 8 tile queue, 2 streamed, 1/4 tiled line sweeps)")
    p.add_argument("--window", type=float, default=0.0, help="tile queue window (0: kernel default)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-batch", action="store_true", help="skip the batched workload in the default run")
    p.add_argument("--workload", default="inverse2048", choices=["inverse2048", "batch256", "appb2048", "adam2048", "softmin"],
                   help="inverse2048: one 2048^2 grid per step (the headline); batch256: 256 grids of sides "
                        "64..1024 per step through rf_batch_solve, with the plain per-grid form beside it; "
                        "adam2048: the inverse problem itself, --adam-steps Adam steps through the autograd "
                        "Function from M = I, w = 0; softmin: the soft-min relaxation (forward, record, adjoint) "
                        "at --size with tau = --tau-rel x h")
    p.add_argument("--tau-rel", type=float, default=0.05)
    p.add_argument("--adam-steps", type=int, default=200)
    p.add_argument("--grids", type=int, default=256)
    return p.parse_args()


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload_config(n):
    return {"workload": f"inverse-problem forward+adjoint step, {n}x{n} FP32 grid",
            "grid": [n, n], "h": 1.0 / (n - 1), "fourier_modes": 16, "drift": "|w|_2 = 0.3 direction field",
            "sources": 4, "observed_fraction": 0.005, "eps": 1e-6, "delta": 0.05,
            "l2": "flushed between timed steps (256 MB write)"}


def sources_sha16(paths):
    import hashlib
    h = hashlib.sha256()
    for p in paths:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """Samples nvidia-smi SM clocks and throttle reasons while running."""

    def __init__(self, index=0):
        self.index = index
        self.samples = []
        self.seen = 0
        self.recording = False
        self._stop = threading.Event()
        self._proc = None

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self._proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                           "--format=csv,noheader,nounits", "-lms", "20"],
                                          stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self._proc = None
            return
        self._t = threading.Thread(target=self._read, daemon=True)
        self._t.start()

    def wait_first(self, timeout=5.0):
        """Block until nvidia-smi delivers samples, then keep only the
        samples taken from now on (the timed region)."""
        t0 = time.time()
        while self._proc and not self.seen and time.time() - t0 < timeout:
            time.sleep(0.05)
        self.recording = True

    def _read(self):
        for line in self._proc.stdout:
            if self._stop.is_set():
                break
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 8:
                self.seen += 1
                if self.recording:
                    self.samples.append(parts)

    def stop(self):
        self._stop.set()
        if self._proc:
            self._proc.terminate()
            try:
                self._proc.wait(timeout=5)
            except Exception:
                self._proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for s in self.samples for k in range(4) if s[4 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


# ---------------------------------------------------------------------------
_REF_INPUT = None


def _oracle_init(n):
    """Pool initialiser: the seeded n x n inputs, generated once per worker."""
    global _REF_INPUT
    import rf_inputs as R
    _REF_INPUT = R.config_inverse(n=n, seed=0)


def _oracle_step(_k=0):
    """One forward+adjoint of the FP64 oracle (single thread) on the worker's
    inputs; returns (seconds, GS iterations)."""
    import oracle as O
    c = _REF_INPUT
    t0 = time.perf_counter()
    out = O.solve_and_grad(c["raw"].astype(np.float64), c["src"], c["h"], c["eps"], c["delta"],
                           c["g"].astype(np.float64))
    return time.perf_counter() - t0, out["iters"]


def oracle_once(n):
    """cpu_baseline: one full n x n forward+adjoint of the oracle on one
    core, timed as it stands (no extrapolation)."""
    _oracle_init(n)
    return _oracle_step()


def run_reference(args):
    """The oracle as the reference arm: every step is one full forward+adjoint
    of the same 2048^2 workload (FP64, the oracle's own GS solve, record and
    reverse-T adjoint).  Steps run one per process on the host's cores (a
    spawn pool started before anything touches a GPU), so K steps take about
    ceil(K / cores) solve times; value = steps / wall time of the timed steps."""
    import multiprocessing as mp
    rank, world, _ = dist_info()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
        if rank != 0:
            dist.barrier()
            return
    cores = os.cpu_count() or 1
    workers = max(1, min(args.steps, cores))
    with mp.get_context("spawn").Pool(workers, initializer=_oracle_init, initargs=(args.size,)) as pool:
        if args.warmup:
            pool.map(_oracle_step, range(args.warmup), chunksize=1)
        t0 = time.perf_counter()
        res = pool.map(_oracle_step, range(args.steps), chunksize=1)
        wall = time.perf_counter() - t0
    value = args.steps / wall
    per_solve = statistics.mean(r[0] for r in res)
    sample = (f"FP64 oracle as it stands: {args.steps} forward+adjoint solves of the {args.size}x{args.size} workload, "
              f"one per process on {workers} host cores ({per_solve:.1f} s per solve on one core, "
              f"{res[0][1]} GS iterations); value = solves / wall time")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": wall / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args.size),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": workers, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def run_ours(args):
    import torch

    import rf_inputs as R
    from paper_2603_00035_gb300 import api
    from paper_2603_00035_gb300 import build as B
    from paper_2603_00035_gb300 import replicas

    rank, world, local = dist_info()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    B.build()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    n = args.size
    c = R.config_inverse(n=n, seed=rank)
    eps, delta, h = c["eps"], c["delta"], c["h"]
    raw = torch.from_numpy(c["raw"]).to(dev)
    src = torch.from_numpy(c["src"]).to(dev)
    g = torch.from_numpy(c["g"]).to(dev)
    ctx = api.Context.get(local)
    tile = {"band": args.band, "block": args.block, "variant": args.variant, "window": args.window,
            "autotuned": False}
    if not args.variant:
        from paper_2603_00035_gb300 import autotune
        proj0, _ = api.rf_project(raw, eps, delta)
        b_, k_, n_, w_ = autotune.tune_sweep(proj0, eps, src, h)
        tile = {"band": b_, "block": k_, "variant": n_, "window": w_, "autotuned": True,
                "cache": autotune.cache_path()}
        del proj0
    opts = api.make_opts(band=tile["band"], block=tile["block"], variant=tile["variant"], window=tile["window"])
    stream = torch.cuda.current_stream()
    # preallocated outputs: the timed steps allocate nothing
    proj = torch.empty_like(raw)
    clip = torch.empty((n, n), dtype=torch.uint8, device=dev)
    T = torch.empty((n, n), dtype=torch.float32, device=dev)
    rec = api.Record.empty(n, n, dev)
    gproj = torch.empty_like(raw)
    lam = torch.empty((n, n), dtype=torch.float32, device=dev)
    graw = torch.empty_like(raw)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]

    def step(events=None):
        if events:
            events[0].record(stream)
        api.rf_project(raw, eps, delta, proj5=proj, clip=clip, ctx=ctx)
        if events:
            events[1].record(stream)
        api.rf_sweep_forward(proj, eps, src, h, opts=opts, T=T, record=False, ctx=ctx)
        if events:
            events[2].record(stream)
        api.rf_record_stencils(proj, eps, src, h, T, rec=rec, ctx=ctx)
        if events:
            events[3].record(stream)
        api.rf_adjoint(src, T, rec, g, algo=args.algo, lam=False, dLdproj5=gproj, ctx=ctx)
        if events:
            events[4].record(stream)
        api.rf_project_backward(raw, clip, eps, delta, gproj, draw5=graw, ctx=ctx)
        if events:
            events[5].record(stream)

    for _ in range(args.warmup):
        step()
    st = ctx.stats()
    if st["status"] != 0:
        raise RuntimeError(f"solver status {st}")
    sweeps, adj_sweeps, cell_updates = st["sweeps"], st["adj_sweeps"], st["cell_updates"]

    phase = np.zeros(5)
    total_ms = 0.0
    sampler = ClockSampler(local)
    sampler.start()
    sampler.wait_first()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush.zero_()
        step(ev)
        torch.cuda.synchronize()
        ph = [ev[i].elapsed_time(ev[i + 1]) for i in range(5)]
        phase += np.array(ph)
        total_ms += ev[0].elapsed_time(ev[5])
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    sampler.stop()
    st = ctx.stats()
    if st["status"] != 0:
        raise RuntimeError(f"solver status {st}")

    # e2e: public API from pinned host buffers, copies inside the timed region
    e2e = None
    if not args.no_e2e:
        # rf_step_host: each step's inputs copied in from pinned host memory,
        # the five phases, T and the raw-field gradient copied back; the
        # library pipelines the copies of neighbouring steps with the compute.
        h_raw = torch.from_numpy(c["raw"]).pin_memory()
        h_src = torch.from_numpy(c["src"]).pin_memory()
        h_g = torch.from_numpy(c["g"]).pin_memory()
        h_T = [torch.empty((n, n), dtype=torch.float32).pin_memory() for _ in range(2)]
        h_graw = [torch.empty((5, n, n), dtype=torch.float32).pin_memory() for _ in range(2)]

        def host_steps(k):
            api.rf_step_host([h_raw] * k, [h_src] * k, [h_g] * k, h, eps, delta,
                             [h_T[i % 2] for i in range(k)], [h_graw[i % 2] for i in range(k)], opts=opts,
                             algo=args.algo, ctx=ctx, stream=stream)

        host_steps(args.warmup)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        host_steps(args.steps)  # returns once the last result is in host memory
        e1.record(stream)
        torch.cuda.synchronize()
        e2e_ms = e0.elapsed_time(e1)
        st = ctx.stats()
        if st["status"] != 0:
            raise RuntimeError(f"solver status {st}")
        h2d = h_raw.numel() * 4 + h_src.numel() + h_g.numel() * 4
        d2h = h_T[0].numel() * 4 + h_graw[0].numel() * 4
        e2e_rate, _ = replicas.job_rate(args.steps, e2e_ms, dev)
        e2e = {"value": e2e_rate, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "how": "one rf_step_host call (C ABI, host buffers) for all steps: each step copies its inputs in "
                      "and T and dL/draw out; the library overlaps the copies of neighbouring steps with the "
                      "compute (two device buffer sets, its own copy streams); no extra L2 flush: each step's "
                      "data arrive by copy, ~400 MB per step"}

    # whole job: the grids all ranks solved over the slowest rank's time
    value, total_ms = replicas.job_rate(args.steps, total_ms, dev)
    ms_per_step = total_ms / args.steps

    phase_ms = phase / args.steps
    names = ["project", "sweep_forward", "record", "adjoint", "project_backward"]
    dom = int(np.argmax(phase_ms))
    peak, peak_kind = measured_peaks()
    if names[dom] == "sweep_forward":
        bytes_per_launch = ALG_BYTES_PER_UPDATE * cell_updates
    elif names[dom] == "adjoint" and args.algo == "sweep":
        # per node per adjoint sweep: id 1 B + w1 4 B + lambda read 4 B + write 4 B + g 4 B + T 4 B
        bytes_per_launch = 21 * adj_sweeps * n * n + 44 * n * n
    elif names[dom] == "adjoint" and args.algo == "levels":
        # levels: two sorts (2 x 16 B per node) + depth pass (id 1, T 4, order 4, state 8 r + 8 w, level 4)
        # + starts 4 + gather (order 4, id 1, w1 4, lambda 4 r + 4 w, g 4, dT 20, grad 20)
        bytes_per_launch = (32 + 29 + 4 + 65) * n * n
    elif names[dom] == "adjoint" and args.algo == "tiles":
        # tiles: tile keys (T 4 B per node; the tile sort is 16384 pairs) + per node id 1 + w1 4 + state
        # 8 r + 8 w + g 4 + T 4 + dT 20 + grad 20
        bytes_per_launch = (4 + 69) * n * n
    elif names[dom] == "adjoint":
        # ordered: sort keys+values (2 x 4 B in, 2 x 4 B out) + per node id 1 + w1 4 + state 8 r + 8 w
        # + g 4 + T 4 + dT 20 + grad 20
        bytes_per_launch = (16 + 69) * n * n
    else:
        bytes_per_launch = 60 * n * n
    achieved = bytes_per_launch / (phase_ms[dom] / 1e3) / 1e9
    traffic = None
    if names[dom] == "sweep_forward" and tile["variant"] in (0, 8) and tile["band"] in (0, 16):
        cap = TRAFFIC_CAPTURES.get(("tile_solve_kernel<16>", n, float(tile["window"] or 4.0)))
        if cap and sources_sha16(TRAFFIC_SOURCES) == cap["sources_sha16"]:
            traffic = cap["bytes"]
    roofline = {"bound": "hbm", "kernel": names[dom], "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": peak_kind, "traffic": traffic}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": dict(workload_config(n), tile=tile),
            "roofline": roofline, "e2e": e2e,
            "gpu_launches": (LAUNCHES_BASE + LAUNCHES_FORWARD[tile["variant"] or 8] + LAUNCHES_ADJOINT[args.algo]) *
                            args.steps,
            "clocks": sampler.summary(),
            "solver": {"sweeps": sweeps, "adj_sweeps": adj_sweeps, "cell_updates": cell_updates,
                       "gcell_updates_per_s": cell_updates / (phase_ms[1] / 1e3) / 1e9,
                       "phase_ms": dict(zip(names, [round(float(x), 4) for x in phase_ms])),
                       "algo": args.algo}}
    if world == 1 and not args.no_batch:
        # the batched workload (256 grids, sides 64..1024) beside the headline:
        # one graph replay per step against the plain per-grid form
        line["batch256"] = batch_measure(batch_grids(args.grids), max(3, args.steps // 2), 2, dev)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        t_solve, iters = oracle_once(n)
        line["cpu_baseline"] = {"value": 1.0 / t_solve, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"FP64 oracle as it stands, one thread: one full forward+adjoint of the "
                                          f"same {n}x{n} workload ({t_solve:.1f} s, {iters} GS iterations), "
                                          f"timed after the GPU steps"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()


def batch_grids(count, seed=0):
    """The batched workload: long side s ~ U{64..1024}, half square, half
    2:1; fields as the 64x64 workload (8 modes, |w| = 0.3); 1-8 sources;
    dL/dT on 1 % of the nodes."""
    import rf_inputs as R
    rng = np.random.default_rng(seed)
    grids = []
    for b, (ny, nx) in enumerate(R.batch_shapes(count, seed)):
        h = 1.0 / (max(ny, nx) - 1)
        grids.append(dict(raw=R.randers_fields(ny, nx, h, 8, seed * 1000 + b, omega="unit", omega_scale=0.3),
                          src=R.random_sources(ny, nx, int(rng.integers(1, 9)), seed * 1000 + b),
                          g=R.sparse_loss_grad(ny, nx, 0.01, b), h=h))
    return grids


def batch_measure(grids, steps, warmup, dev, world=1, sampler=None, variant=0):
    """Time the batched workload through one CUDA-graph replay of
    BatchSolver (rf_project, rf_batch_solve, rf_project_backward) and, beside
    it, the plain form: the same grids one by one through the single-grid
    entry points.  Returns the result dict (rates for this rank's grids)."""
    import torch

    from paper_2603_00035_gb300 import api
    from paper_2603_00035_gb300 import replicas

    bs = api.BatchSolver(grids, opts=api.make_opts(variant=variant))
    tuned = None
    if not variant:
        from paper_2603_00035_gb300 import autotune
        tuned = autotune.tune_batch(bs)
    bs.run()
    torch.cuda.synchronize()
    bs.capture()
    for _ in range(warmup):
        bs.run()
    torch.cuda.synchronize()
    st = api.Context.get(dev).stats()
    if st["status"] != 0 or int(bs.gstat[:, 0].abs().sum()) != 0:
        raise RuntimeError(f"batch status {st}, per-grid {bs.gstat[:, 0].tolist()}")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if sampler:
        sampler.start()
        sampler.wait_first()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0.record()
    for _ in range(steps):
        bs.run()
    e1.record()
    torch.cuda.synchronize()
    if sampler:
        sampler.stop()
    rate, total = replicas.job_rate(len(grids) * steps, e0.elapsed_time(e1), dev)
    sweeps = bs.gstat[:, 1].double().mean().item()
    per = []
    for g in grids:
        per.append((torch.from_numpy(g["raw"]).to(dev), torch.from_numpy(g["src"]).to(dev),
                    torch.from_numpy(g["g"]).to(dev), g["h"]))

    def plain():
        for raw, src, gg, h in per:
            proj, clip = api.rf_project(raw, 1e-6, 0.05)
            T, rec = api.rf_sweep_forward(proj, 1e-6, src, h)
            gproj, _ = api.rf_adjoint(src, T, rec, gg, algo="tiles", lam=False)
            api.rf_project_backward(raw, clip, 1e-6, 0.05, gproj)

    plain()
    torch.cuda.synchronize()
    e0.record()
    plain()
    e1.record()
    torch.cuda.synchronize()
    plain_rate, plain_ms = replicas.job_rate(len(grids), e0.elapsed_time(e1), dev)
    nodes = sum(g["src"].size for g in grids)
    return {"value": rate, "unit": UNIT, "ms_per_batch": total / steps, "grids": len(grids), "nodes": int(nodes),
            "mean_forward_sweep_equivalents": sweeps, "steps": steps, "warmup": warmup,
            "how": "one CUDA-graph replay of rf_project + rf_batch_solve + rf_project_backward (variant, tile side "
                   "and window from the batch autotuner unless given)",
            "plain_form": {"value": plain_rate, "unit": UNIT, "ms_per_batch": plain_ms,
                           "how": "rf_project, rf_sweep_forward, rf_adjoint (tiles), rf_project_backward per grid"},
            "speedup_vs_plain": rate / plain_rate,
            "autotuned": None if tuned is None else {"band": tuned[0], "variant": tuned[1], "window": tuned[2]}}


def run_batch(args):
    import torch

    from paper_2603_00035_gb300 import build as B
    from paper_2603_00035_gb300 import replicas

    rank, world, local = dist_info()
    if world > 1:
        torch.distributed.init_process_group("nccl")
    B.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    all_grids = batch_grids(args.grids)
    # independent grids shard with no data exchange: each rank solves its own
    # size-balanced subset
    grids = [all_grids[i] for i in replicas.shard([g["src"].size for g in all_grids], rank, world)]
    nodes = sum(g["src"].size for g in all_grids)
    sampler = ClockSampler(local)
    res = batch_measure(grids, args.steps, args.warmup, dev, world, sampler, args.variant)
    line = {"metric": f"forward+adjoint solves/s, batch of {len(all_grids)} grids (sides 64..1024)",
            "value": res["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": res["ms_per_batch"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"batched forward+adjoint, {len(all_grids)} grids, long side U{{64..1024}}, "
                                   "half square / half 2:1, 1-8 sources, CUDA-graph replay",
                       "nodes": int(nodes), "mean_sweeps": res["mean_forward_sweep_equivalents"],
                       "l2": "working set > L2 (%.0f MB of fields)" % (nodes * 20 / 1e6)},
            "plain_form": res["plain_form"],
            # per replay: project, init, plan, tile map, reset, seed, finish-seed, solve, stats, record,
            # adjoint-status column, sort keys, gather, unreached, project backward (CUB's sort not counted)
            "gpu_launches": 15 * args.steps,
            "clocks": sampler.summary()}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()


def run_appb(args):
    """The paper's own parameterisation layers (App. B) at n x n: eigenvalue-
    clamp projection into the solver's factor form, Log-Euclidean + drift TV
    with gradient, and the projection backward -- one regularised projection
    pass per step.  Each kernel is timed with CUDA events on the launching
    stream; algorithmic bytes per node: projection 20 B read + 40 B written,
    TV 20 B read + 40 B gradient read-modify-write, backward 60 B read + 20 B
    written."""
    import torch

    import rf_inputs as R
    from paper_2603_00035_gb300 import api
    from paper_2603_00035_gb300 import build as B

    B.build()
    torch.cuda.set_device(0)
    n = args.size
    dev = torch.device("cuda")
    gb = torch.from_numpy(R.gb_fields(n, n, 1.0 / (n - 1), 16, 0)).to(dev)
    prm = api.metric_params(0.5, 3.0, 1.2, 0.1, 1e-6)
    gbp, proj = torch.empty_like(gb), torch.empty_like(gb)
    grad = torch.zeros_like(gb)
    dproj = torch.randn(gb.shape, device=dev, generator=torch.Generator(device=dev).manual_seed(1))
    dgb = torch.empty_like(gb)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2
    s = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    names = ["rf_metric_project", "rf_tv", "rf_metric_project_backward"]
    times = {k: [] for k in names}

    def step(timed):
        if timed:
            ev[0].record(s)
        api.rf_metric_project(gb, prm, gbp5=gbp, proj5=proj)
        if timed:
            ev[1].record(s)
        api.rf_tv(gbp, "log_euclidean", 1e-3, 1e-3, grad5=grad, value=True)
        if timed:
            ev[2].record(s)
        api.rf_metric_project_backward(gb, prm, dproj5=dproj, dgbp5=grad, dgb5=dgb)
        if timed:
            ev[3].record(s)

    for _ in range(args.warmup):
        step(False)
    torch.cuda.synchronize()
    if api.Context.get(0).stats()["status"] != 0:
        raise RuntimeError("App. B layers reported a device error")
    sampler = ClockSampler(0)
    sampler.start()
    sampler.wait_first()
    total = 0.0
    for _ in range(args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        step(True)
        torch.cuda.synchronize()
        for k, name in enumerate(names):
            times[name].append(ev[k].elapsed_time(ev[k + 1]))
        total += ev[0].elapsed_time(ev[3])
    sampler.stop()
    peak, kind = measured_peaks()
    nodes = n * n
    bytes_per_node = {"rf_metric_project": 60, "rf_tv": 60, "rf_metric_project_backward": 80}
    kern = {}
    for name in names:
        ms = statistics.mean(times[name])
        gbs = bytes_per_node[name] * nodes / (ms * 1e-3) / 1e9
        kern[name] = {"ms": ms, "achieved_gbs": gbs, "frac": gbs / peak, "bytes_per_node": bytes_per_node[name]}
    top = max(names, key=lambda k: kern[k]["ms"])
    ms_step = total / args.steps
    line = {"metric": f"App. B regularised projection passes/s at {n}x{n}", "value": 1e3 / ms_step,
            "unit": "passes/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"eigenvalue-clamp projection + Log-Euclidean/drift TV + backward, {n}x{n}",
                       "fields": "gb_fields, 16 modes, eigenvalues 0.25..4, |b| up to 1.5",
                       "params": "lam 0.5..3, b_max 1.2, delta 0.1",
                       "l2": "flushed between timed steps (256 MB write)"},
            "roofline": {"bound": "hbm", "kernel": top, "achieved": kern[top]["achieved_gbs"], "peak": peak,
                         "unit": "GB/s", "frac": kern[top]["frac"], "traffic": None, "peak_kind": kind},
            "kernels": kern, "gpu_launches": 4 * args.steps, "clocks": sampler.summary()}
    print(json.dumps(line), flush=True)


def run_adam(args):
    """The inverse metric problem at n x n (Sec. 4, Eq. 8): recover the five
    fields (L11, L21, L22, wx, wy) of a 16-mode ground truth from arrival
    times observed on 0.5 % of the nodes, with Adam (1e-2 on L, 5e-3 on w)
    through RFSolve, from M = I, w = 0.  Reports the loss and the relative
    recovery errors of the metric and the drift."""
    import torch

    import rf_inputs as R
    from paper_2603_00035_gb300 import build as B
    from paper_2603_00035_gb300.inverse import run_inverse

    B.build()
    torch.cuda.set_device(0)
    n = args.size
    c = R.config_inverse(n=n, seed=0)
    raw_true = torch.from_numpy(c["raw"]).cuda()
    src = torch.from_numpy(c["src"]).cuda()
    obs = torch.from_numpy(c["obs"]).cuda()
    run_inverse(raw_true, src, obs, c["h"], steps=3)  # warm-up: builds, workspace
    torch.cuda.synchronize()
    out = run_inverse(raw_true, src, obs, c["h"], steps=args.adam_steps, log_every=max(1, args.adam_steps // 10))
    hist = out["loss_history"]
    line = {"metric": f"inverse problem {n}x{n}: Adam steps/s through RFSolve", "value": out["steps"] / out["seconds"],
            "unit": "steps/s", "n_gpus": 1, "steps": out["steps"], "warmup": 3,
            "ms_per_step": 1e3 * out["seconds"] / out["steps"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"inverse metric problem {n}x{n}, 16-mode ground truth, 4 sources, "
                                   f"{100 * c['obs'].mean():.2f} % observed, Adam lr 1e-2 (L) / 5e-3 (w), "
                                   "initial M = I, w = 0", "steps": out["steps"]},
            "loss_first": hist[0][1], "loss_last_logged": hist[-1][1], "final_loss": out["final_loss"],
            "loss_history": hist, "rel_err_metric": out["rel_err_metric"], "rel_err_drift": out["rel_err_drift"],
            "timing": "wall clock of the whole Adam loop (forward, backward, optimiser), synchronised at the end"}
    print(json.dumps(line), flush=True)


def run_softmin(args):
    """Forward + record + adjoint of the soft-min relaxation on the n x n
    inverse-problem workload, tau = tau_rel x h; CUDA events per phase, L2
    flushed between steps."""
    import torch

    import rf_inputs as R
    from paper_2603_00035_gb300 import api
    from paper_2603_00035_gb300 import build as B

    B.build()
    torch.cuda.set_device(0)
    n = args.size
    c = R.config_inverse(n=n, seed=0)
    tau = args.tau_rel * c["h"]
    raw = torch.from_numpy(c["raw"]).cuda()
    src = torch.from_numpy(c["src"]).cuda()
    g = torch.from_numpy(c["g"]).cuda()
    ctx = api.Context.get(0)
    proj, _ = api.rf_project(raw, c["eps"], c["delta"])
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    # forward: the tile queue with the soft-min update (variant 0 / 8), or a
    # line-sweep variant's number for Jacobi iterations over the whole grid
    sopts = api.make_opts(variant=args.variant)
    tile_fwd = args.variant in (0, 8)

    def step(timed):
        if timed:
            ev[0].record()
        T = api.rf_softmin_forward(proj, c["eps"], src, c["h"], tau, opts=sopts)
        if timed:
            ev[1].record()
        wnb, dT = api.rf_softmin_record(proj, c["eps"], src, c["h"], T, tau)
        if timed:
            ev[2].record()
        api.rf_softmin_adjoint(src, T, wnb, dT, g, lam=False)
        if timed:
            ev[3].record()

    for _ in range(args.warmup):
        step(False)
    st = ctx.stats()
    if st["status"] != 0:
        raise RuntimeError(f"soft-min status {st}")
    iters, adj = st["sweeps"], st["adj_sweeps"]
    ph = np.zeros(3)
    for _ in range(args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        step(True)
        torch.cuda.synchronize()
        ph += np.array([ev[k].elapsed_time(ev[k + 1]) for k in range(3)])
    ph /= args.steps
    ms = float(ph.sum())
    line = {"metric": f"soft-min forward+adjoint solves/s at {n}x{n}", "value": 1e3 / ms, "unit": "solves/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"soft-min relaxation, {n}x{n} inverse-problem fields, tau = {args.tau_rel} h",
                       "l2": "flushed between timed steps (256 MB write)"},
            "phase_ms": {"forward": ph[0], "record": ph[1], "adjoint": ph[2]},
            "forward": "tile queue" if tile_fwd else "Jacobi over the grid",
            "forward_sweeps": iters, "adjoint_iterations": adj,
            "gpu_launches": (10 if tile_fwd else 5) * args.steps}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch256":
        run_batch(args)
    elif args.workload == "appb2048":
        run_appb(args)
    elif args.workload == "adam2048":
        run_adam(args)
    elif args.workload == "softmin":
        run_softmin(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
