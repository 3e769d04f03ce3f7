"""Command-line timing of one forward solve on the inverse-problem workload.

    python -m paper_2603_00035_gb300.solve --size 2048 --variant tiles --band 16 --repeat 3

builds the seeded n x n workload (16-mode Fourier metric, |w| = 0.3 drift,
4 sources), projects it, runs rf_sweep_forward `repeat` times and prints one
JSON line per solve: CUDA-event milliseconds and the solver statistics
(rounds of the tile queue, node updates, status).  Every step runs in
librf's kernels.
"""
from __future__ import annotations

import argparse
import json
import os
import sys


def main(argv=None):
    p = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    p.add_argument("--size", type=int, default=2048)
    p.add_argument("--variant", default="auto", help="auto, tiles, streamed, tiled1, tiled4")
    p.add_argument("--band", type=int, default=0, help="tile side (tiles) or band (line sweeps); 0 = auto")
    p.add_argument("--block", type=int, default=0)
    p.add_argument("--window", type=float, default=0.0)
    p.add_argument("--rtol", type=float, default=1e-6)
    p.add_argument("--repeat", type=int, default=3)
    p.add_argument("--record", action="store_true", help="also write the stencil record")
    a = p.parse_args(argv)
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch

    import rf_inputs as R
    from . import api
    from . import build as B

    B.build()
    c = R.config_inverse(n=a.size, seed=0)
    raw = torch.from_numpy(c["raw"]).cuda()
    src = torch.from_numpy(c["src"]).cuda()
    proj, _ = api.rf_project(raw, c["eps"], c["delta"])
    ctx = api.Context.get(0)
    o = api.make_opts(variant=a.variant, band=a.band, block=a.block, window=a.window, rtol=a.rtol)
    T = torch.empty_like(src, dtype=torch.float32)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for k in range(a.repeat):
        e0.record()
        api.rf_sweep_forward(proj, c["eps"], src, c["h"], opts=o, T=T, record=a.record)
        e1.record()
        st = ctx.stats()
        print(json.dumps(dict(solve=k, ms=e0.elapsed_time(e1), status=st["status_name"], rounds=st["rounds"],
                              sweeps=st["sweeps"], node_updates=st["cell_updates"])), flush=True)
        if st["status"] != 0:
            raise SystemExit(1)


if __name__ == "__main__":
    main()
