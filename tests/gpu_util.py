"""Helpers shared by the GPU parity tests: build/load the CUDA library, run
the whole CUDA path and the FP64 oracle on the same seeded inputs, and the
tolerance rules.

Tolerances (the parity bar):
* forward: max |T_gpu - T_oracle| <= 1e-4 * max T over reached nodes, and
  the reached set identical;
* gradients: relative L2 <= 1e-3 over nodes outside the flip set;
* flip set: nodes whose stencil id differs between GPU and oracle, or whose
  oracle best-vs-second valid candidate margin is < 1e-5 * max T.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_2603_00035_gb300 import api  # noqa: E402
from paper_2603_00035_gb300 import build as B  # noqa: E402

FWD_TOL = 1e-4
GRAD_TOL = 1e-3
FLIP_MARGIN = 1e-5


def require_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()


def to_dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def gpu_path(raw, src, h, eps, delta, g, opts=None, algo="sweep"):
    """project -> forward (+record) -> adjoint -> project backward on the GPU."""
    raw_t = to_dev(raw, torch.float32)
    src_t = to_dev(src, torch.uint8)
    g_t = to_dev(g, torch.float32)
    ctx = api.Context.get(0)
    proj, clip = api.rf_project(raw_t, eps, delta)
    T, rec = api.rf_sweep_forward(proj, eps, src_t, h, opts=opts)
    st_fwd = ctx.stats()
    gproj, lam = api.rf_adjoint(src_t, T, rec, g_t, algo=algo)
    graw = api.rf_project_backward(raw_t, clip, eps, delta, gproj)
    st_adj = ctx.stats()
    out = dict(proj=proj, clip=clip, T=T, rec=rec, gproj=gproj, lam=lam, graw=graw, st_fwd=st_fwd,
               st_adj=st_adj)
    return {k: (v.cpu().numpy() if isinstance(v, torch.Tensor) else v) for k, v in out.items()} | \
        dict(rec_np=dict(id=rec.id.cpu().numpy(), w1=rec.w1.cpu().numpy(), dT=rec.dT.cpu().numpy()))


def oracle_path(raw, src, h, eps, delta, g):
    return O.solve_and_grad(np.asarray(raw, np.float64), src, h, eps, delta, np.asarray(g, np.float64))


def flip_mask(gpu, orc):
    T = orc["T"]
    tmax = T[np.isfinite(T)].max()
    flips = (gpu["rec_np"]["id"] != orc["rec"]["id"]) | (orc["rec"]["margin"] < FLIP_MARGIN * tmax)
    return flips, tmax


def rel_l2(a, b, mask=None):
    if mask is not None:
        a, b = a[..., mask], b[..., mask]
    den = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (den if den > 0 else 1.0)
