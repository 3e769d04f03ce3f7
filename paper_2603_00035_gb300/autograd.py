"""torch.autograd.Function over the solver path.

Forward:  raw (L11, L21, L22, wx, wy) --rf_project--> proj --rf_sweep_forward--> T
Backward: dL/dT --rf_adjoint--> dL/dproj --rf_project_backward--> dL/draw

Implicit differentiation of the converged discrete system (Sec. 3.3,
Eqs. 4-6; Alg. 2): the saved state is T, the stencil record (ids, donor
weights, closed-form partials), the raw fields and the clip mask -- not the
sweep history -- so memory is O(nodes) whatever the sweep count.  Every
step runs in librf's CUDA kernels; this module only wires them to autograd.
"""
from __future__ import annotations

import torch

from . import api


class RFSolve(torch.autograd.Function):
    """T = RFSolve.apply(raw5, src, h, eps, delta, algo, opts).

    raw5: float32 CUDA tensor (5, ny, nx) of L11, L21, L22, wx, wy (the
    projection makes the metric SPD and the drift feasible);
    src: uint8 (ny, nx) source mask.  Returns T (ny, nx), +inf where
    unreached.  Gradients flow to raw5 only.
    """

    @staticmethod
    def forward(ctx, raw5, src, h, eps=1e-6, delta=0.05, algo="ordered", opts=None):
        raw5 = raw5.contiguous()
        proj, clip = api.rf_project(raw5, eps, delta)
        T, rec = api.rf_sweep_forward(proj, eps, src, h, opts=opts)
        ctx.save_for_backward(raw5, clip, src, T, rec.id, rec.w1, rec.dT)
        ctx.cfg = (eps, delta, algo)
        return T

    @staticmethod
    def backward(ctx, gT):
        raw5, clip, src, T, rid, rw1, rdT = ctx.saved_tensors
        eps, delta, algo = ctx.cfg
        g = torch.nan_to_num(gT.contiguous().to(torch.float32), nan=0.0, posinf=0.0, neginf=0.0)
        rec = api.Record(rid, rw1, rdT)
        gproj, _ = api.rf_adjoint(src, T, rec, g, algo=algo, lam=False)
        graw = api.rf_project_backward(raw5, clip, eps, delta, gproj)
        return graw, None, None, None, None, None, None


def rf_solve(raw5, src, h, eps=1e-6, delta=0.05, algo="ordered", opts=None):
    """Differentiable arrival times T(raw5) (see RFSolve)."""
    return RFSolve.apply(raw5, src, h, eps, delta, algo, opts)
