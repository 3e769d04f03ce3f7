"""Helpers shared by the GPU parity tests: build/load the CUDA library, run
the whole CUDA path and the FP64 oracle on the same seeded inputs, and the
tolerance rules.

Tolerances (the parity bar):
* forward: max |T_gpu - T_oracle| <= 1e-4 * max T over reached nodes, and
  the reached set identical;
* gradients: relative L2 <= 1e-3 over nodes outside the flip set;
* stencils are compared in canonical form: a two-point update whose donor
  weight is within DEGENERATE of 1 (or 0) is the one-point update through its
  first (second) donor -- same value to second order, same partials to first
  order -- so the two namings of one update are not a mismatch (FP32 errors
  of ~1e-6 T in the donor times move a barycentric weight by ~1e-6 T / (h
  |m|_M), a few 1e-4 at 1024^2, hence DEGENERATE = 1e-3);
* near-tie: the oracle's best-vs-second valid candidate margin is
  < 1e-5 * max T + 2 e, e the largest |T_gpu - T_oracle| over the node's 3 x 3
  neighbourhood: a candidate is 1-Lipschitz in its donor times (weights in
  [0, 1] summing to 1), so forward errors of e can reorder candidates closer
  than 2 e, and FP32 may legitimately pick either of them;
* flip set: nodes whose canonical stencils differ; every flip must be a
  near-tie (a mismatch outside the near-ties fails), flips are excluded from
  the gradient comparison and their fraction is bounded per workload.
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
DEGENERATE = 1e-3


def require_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()


def to_dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def gpu_path(raw, src, h, eps, delta, g, opts=None, algo="tiles"):
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


def canonical_stencil(ids, w1, with_weight=False):
    """Record ids with degenerate two-point updates renamed to the one-point
    update they equal: 0x20|k with w1 >= 1 - DEGENERATE -> 0x10|k, with
    w1 <= DEGENERATE -> 0x10|((k + 1) % 8).  with_weight: also the donor
    weight in the same form (1 for a renamed update, as for a one-point)."""
    ids = np.asarray(ids).astype(np.int32)
    w1 = np.asarray(w1)
    two = (ids & 0xF0) == 0x20
    k = ids & 7
    hi, lo = two & (w1 >= 1.0 - DEGENERATE), two & (w1 <= DEGENERATE)
    out = np.where(hi, 0x10 | k, ids)
    out = np.where(lo, 0x10 | ((k + 1) & 7), out)
    if with_weight:
        return out, np.where(hi | lo, 1.0, w1)
    return out


def describe_mismatch(mask, gpu_id, gpu_w1, gpu_T, orc_rec, orc_T, limit=6):
    """Text dump of the first nodes of `mask` (for assertion messages)."""
    tmax = orc_T[np.isfinite(orc_T)].max()
    le = local_error(gpu_T, orc_T)
    rows = []
    for i, j in np.argwhere(mask)[:limit]:
        rows.append(f"({i},{j}) gpu id {int(gpu_id[i, j]):#x} w1 {float(gpu_w1[i, j]):.5f} T {float(gpu_T[i, j]):.7g}"
                    f" | oracle id {int(orc_rec['id'][i, j]):#x} w1 {float(orc_rec['w1'][i, j]):.5f}"
                    f" T {float(orc_T[i, j]):.7g} margin/maxT {float(orc_rec['margin'][i, j]) / tmax:.2e}"
                    f" local err/maxT {float(le[i, j]) / tmax:.2e}")
    return "\n".join(rows)


def local_error(T_gpu, T_orc):
    """max |T_gpu - T_oracle| over each node's 3 x 3 neighbourhood (0 where
    both are +inf)."""
    with np.errstate(invalid="ignore"):
        e = np.abs(np.asarray(T_gpu, np.float64) - np.asarray(T_orc, np.float64))
    e = np.where(np.isfinite(e), e, 0.0)
    p = np.pad(e, 1)
    ny, nx = e.shape
    return np.max([p[1 + di:1 + di + ny, 1 + dj:1 + dj + nx] for di in (-1, 0, 1) for dj in (-1, 0, 1)], axis=0)


_DX = (-1, -1, -1, 0, 1, 1, 1, 0)
_DY = (1, 0, -1, -1, -1, 0, 1, 1)


def gpu_choice_is_near_tie(i, j, gid, T_orc, proj, h, eps, bound):
    """The GPU's stencil at node (i, j), evaluated by the oracle's FP64 local
    update at the oracle's T: a near-tie when it is geometrically valid
    (real root, barycentric weights >= 0), its donors precede its value up
    to `bound` (the causality test can flip within the forward error), and
    its value is within `bound` of the oracle's best.  The oracle's margin
    only counts candidates valid at its own T, so a candidate rejected by a
    hair never enters it."""
    ny, nx = T_orc.shape
    Tn = np.array([T_orc[i + _DY[n], j + _DX[n]] if 0 <= i + _DY[n] < ny and 0 <= j + _DX[n] < nx else np.inf
                   for n in range(8)])
    l11, l21, l22, wx, wy = (float(proj[c, i, j]) for c in range(5))
    c = O.cell_eval(Tn, h, l11 * l11 + eps, l11 * l21, l21 * l21 + l22 * l22 + eps, wx, wy)
    k = int(gid) & 7
    if (int(gid) & 0xF0) == 0x20:
        val = c["two"][k]
        ok = np.isfinite(val) and (c["lam"][k] >= 0).all() and max(Tn[k], Tn[(k + 1) & 7]) < val + bound
    elif (int(gid) & 0xF0) == 0x10:
        val = c["one"][k]
        ok = bool(c["one_ok"][k]) and Tn[k] < val + bound
    else:
        return False
    return bool(ok and val <= T_orc[i, j] + bound)


def stencil_compare(gpu_id, gpu_w1, orc_rec, tmax, T_gpu=None, T_orc=None, fields=None):
    """(flips, hard): flips = canonical stencils differ; hard = flips that
    are not near-ties of the oracle (must be empty).  With both T given, the
    near-tie margin includes twice the local forward error; with fields =
    (proj5 FP64, h, eps) as well, a remaining mismatch is re-examined with
    the oracle's own local update (gpu_choice_is_near_tie)."""
    a = canonical_stencil(gpu_id, gpu_w1)
    b = canonical_stencil(orc_rec["id"], orc_rec["w1"])
    flips = a != b
    bound = FLIP_MARGIN * tmax
    if T_gpu is not None and T_orc is not None:
        bound = bound + 2.0 * local_error(T_gpu, T_orc)
    hard = flips & (orc_rec["margin"] >= bound)
    if fields is not None and T_orc is not None and hard.any():
        proj, h, eps = fields
        bnd = np.broadcast_to(bound, hard.shape)
        for i, j in np.argwhere(hard):
            if gpu_choice_is_near_tie(i, j, gpu_id[i, j], T_orc, proj, h, eps, float(bnd[i, j])):
                hard[i, j] = False
    return flips, hard


def flip_mask(gpu, orc):
    T = orc["T"]
    tmax = T[np.isfinite(T)].max()
    flips, _ = stencil_compare(gpu["rec_np"]["id"], gpu["rec_np"]["w1"], orc["rec"], tmax)
    return flips, tmax


def rel_l2(a, b, mask=None):
    if mask is not None:
        a, b = a[..., mask], b[..., mask]
    den = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (den if den > 0 else 1.0)
