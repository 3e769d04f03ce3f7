"""torch.autograd.Function over the solver path.

Forward:  raw (L11, L21, L22, wx, wy) --rf_project--> proj --rf_sweep_forward--> T
Backward: dL/dT --rf_adjoint--> dL/dproj --rf_project_backward--> dL/draw

Implicit differentiation of the converged discrete system (Sec. 3.3,
Eqs. 4-6; Alg. 2): the saved state is T, the stencil record (ids, donor
weights, closed-form partials), the raw fields and the clip mask -- not the
sweep history -- so memory is O(nodes) whatever the sweep count.  Every
step runs in librf's CUDA kernels; this module only wires them to autograd.

Device-detected errors are not silent: after the forward solve and after the
adjoint the context's status word is read (which synchronises the stream),
and a non-converged solve, an expired device wait, a non-finite input or an
empty source mask raises RFError instead of returning gradients of an
unusable T.
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
    def forward(ctx, raw5, src, h, eps=1e-6, delta=0.05, algo="tiles", opts=None):
        raw5 = raw5.contiguous()
        proj, clip = api.rf_project(raw5, eps, delta)
        T, rec = api.rf_sweep_forward(proj, eps, src, h, opts=opts)
        api.Context.get(raw5.device).raise_on_device_error("RFSolve.forward")
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
        api.Context.get(raw5.device).raise_on_device_error("RFSolve.backward")
        return graw, None, None, None, None, None, None


def rf_solve(raw5, src, h, eps=1e-6, delta=0.05, algo="tiles", opts=None):
    """Differentiable arrival times T(raw5) (see RFSolve)."""
    return RFSolve.apply(raw5, src, h, eps, delta, algo, opts)


class SoftSolve(torch.autograd.Function):
    """T = SoftSolve.apply(raw5, src, h, tau, eps, delta, opts): the
    soft-min relaxation of the solver (Sec. 3.3; each node takes -tau log
    sum_k exp(-c_k / tau) over its 8 stencil segment minima), differentiated
    through its own record and adjoint.  Device errors raise RFError."""

    @staticmethod
    def forward(ctx, raw5, src, h, tau, eps=1e-6, delta=0.05, opts=None):
        raw5 = raw5.contiguous()
        proj, clip = api.rf_project(raw5, eps, delta)
        T = api.rf_softmin_forward(proj, eps, src, h, tau, opts=opts)
        wnb, dT = api.rf_softmin_record(proj, eps, src, h, T, tau)
        api.Context.get(raw5.device).raise_on_device_error("SoftSolve.forward")
        ctx.save_for_backward(raw5, clip, src, T, wnb, dT)
        ctx.cfg = (eps, delta)
        return T

    @staticmethod
    def backward(ctx, gT):
        raw5, clip, src, T, wnb, dT = ctx.saved_tensors
        eps, delta = ctx.cfg
        g = torch.nan_to_num(gT.contiguous().to(torch.float32), nan=0.0, posinf=0.0, neginf=0.0)
        gproj, _ = api.rf_softmin_adjoint(src, T, wnb, dT, g, lam=False)
        graw = api.rf_project_backward(raw5, clip, eps, delta, gproj)
        api.Context.get(raw5.device).raise_on_device_error("SoftSolve.backward")
        return graw, None, None, None, None, None, None


# ---- the paper's own parameterisation (App. B) ---------------------------------

class MetricProject(torch.autograd.Function):
    """(gbp5, proj5) = MetricProject.apply(gb5, prm): App. B projection of
    (g11, g12, g22, b1, b2) -- eigenvalue clamp, drift clip and G^-1-norm
    rescale -- and the solver's factor form.  Backward recomputes from gb5."""

    @staticmethod
    def forward(ctx, gb5, prm):
        gb5 = gb5.contiguous()
        gbp5, proj5 = api.rf_metric_project(gb5, prm)
        ctx.save_for_backward(gb5)
        ctx.prm = prm
        return gbp5, proj5

    @staticmethod
    def backward(ctx, dgbp5, dproj5):
        (gb5,) = ctx.saved_tensors
        dgbp5 = dgbp5.contiguous() if dgbp5 is not None else None
        dproj5 = dproj5.contiguous() if dproj5 is not None else None
        return api.rf_metric_project_backward(gb5, ctx.prm, dproj5=dproj5, dgbp5=dgbp5), None


class SweepSolve(torch.autograd.Function):
    """T = SweepSolve.apply(proj5, src, h, eps, algo, opts): the solve of an
    already-feasible factor-form field (no projection), differentiated by the
    stencil-record adjoint (Alg. 2)."""

    @staticmethod
    def forward(ctx, proj5, src, h, eps=1e-6, algo="tiles", opts=None):
        proj5 = proj5.contiguous()
        T, rec = api.rf_sweep_forward(proj5, eps, src, h, opts=opts)
        api.Context.get(proj5.device).raise_on_device_error("SweepSolve.forward")
        ctx.save_for_backward(src, T, rec.id, rec.w1, rec.dT)
        ctx.algo = algo
        return T

    @staticmethod
    def backward(ctx, gT):
        src, T, rid, rw1, rdT = ctx.saved_tensors
        g = torch.nan_to_num(gT.contiguous().to(torch.float32), nan=0.0, posinf=0.0, neginf=0.0)
        gproj, _ = api.rf_adjoint(src, T, api.Record(rid, rw1, rdT), g, algo=ctx.algo, lam=False)
        api.Context.get(T.device).raise_on_device_error("SweepSolve.backward")
        return gproj, None, None, None, None, None


class TotalVariation(torch.autograd.Function):
    """w_metric R(G) + w_drift R(b) of App. B (metric: "frobenius",
    "log_euclidean" or "none") as a 0-d tensor."""

    @staticmethod
    def forward(ctx, gb5, metric="frobenius", w_metric=1.0, w_drift=1.0):
        gb5 = gb5.contiguous()
        val, _ = api.rf_tv(gb5, metric)
        ctx.save_for_backward(gb5)
        ctx.cfg = (metric, w_metric, w_drift)
        return w_metric * val[0] + w_drift * val[1]

    @staticmethod
    def backward(ctx, gout):
        (gb5,) = ctx.saved_tensors
        metric, wm, wd = ctx.cfg
        grad = torch.zeros_like(gb5)
        api.rf_tv(gb5, metric, wm, wd, grad5=grad, value=False)
        return grad * gout, None, None, None


def metric_solve(gb5, src, h, prm, algo="tiles", opts=None):
    """Differentiable T of the paper's raw (g11, g12, g22, b1, b2) fields:
    App. B projection, then the solve.  Returns (T, gbp5)."""
    gbp5, proj5 = MetricProject.apply(gb5, prm)
    return SweepSolve.apply(proj5, src, h, prm.eps, algo, opts), gbp5
