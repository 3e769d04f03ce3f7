"""Thin PyTorch-facing wrappers with the names of the C ABI (include/rf.h).

PyTorch supplies device memory and the current stream; every step of the
solver runs in librf's CUDA kernels.  Functions take and return CUDA
tensors: float32 5-plane fields of shape (5, ny, nx), uint8 masks (ny, nx).
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import torch

from . import _lib as L


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _check_cuda(t, dtype, shape=None, name="tensor"):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")


class Context:
    """Owns one rf_ctx (workspace + device status word) on one device."""

    _by_device: dict = {}

    def __init__(self, device: int = 0):
        lib = L.load()
        self.device = device
        self.handle = ctypes.c_void_p()
        L.check(lib.rf_ctx_create(ctypes.byref(self.handle), device), "rf_ctx_create")

    @classmethod
    def get(cls, device=None) -> "Context":
        if device is None:
            device = torch.cuda.current_device()
        if isinstance(device, torch.device):
            device = device.index if device.index is not None else torch.cuda.current_device()
        if device not in cls._by_device:
            cls._by_device[device] = Context(device)
        return cls._by_device[device]

    def set_timeout(self, ns: int):
        L.check(L.load().rf_ctx_set_timeout(self.handle, int(ns)), "rf_ctx_set_timeout")

    def stats(self) -> dict:
        st = L.Stats()
        L.load().rf_ctx_last_stats(self.handle, ctypes.byref(st))
        return dict(status=st.status, status_name=L.STATUS.get(st.status, str(st.status)), sweeps=st.sweeps,
                    converged=bool(st.converged), adj_sweeps=st.adj_sweeps, cell_updates=st.cell_updates,
                    max_residual=st.max_residual)

    def __del__(self):
        try:
            if self.handle:
                L.load().rf_ctx_destroy(self.handle)
        except Exception:
            pass


@dataclass
class Record:
    """Per-node record of the converged forward solve (rf_record)."""
    id: torch.Tensor   # uint8 (ny, nx)
    w1: torch.Tensor   # float32 (ny, nx)
    dT: torch.Tensor   # float32 (5, ny, nx)

    def c(self):
        return L.Record(self.id.data_ptr(), self.w1.data_ptr(), self.dT.data_ptr())

    @staticmethod
    def empty(ny, nx, device):
        return Record(torch.empty((ny, nx), dtype=torch.uint8, device=device),
                      torch.empty((ny, nx), dtype=torch.float32, device=device),
                      torch.empty((5, ny, nx), dtype=torch.float32, device=device))


def _grid(ny, nx, h):
    return L.Grid(int(ny), int(nx), float(h))


def rf_project(raw5, eps, delta, proj5=None, clip=None, ctx=None, stream=None):
    """a1: M = L L^T + eps I; w scaled to |w|_{M^-1} <= 1 - delta."""
    _check_cuda(raw5, torch.float32, name="raw5")
    _, ny, nx = raw5.shape
    ctx = ctx or Context.get(raw5.device)
    proj5 = proj5 if proj5 is not None else torch.empty_like(raw5)
    clip = clip if clip is not None else torch.empty((ny, nx), dtype=torch.uint8, device=raw5.device)
    g = _grid(ny, nx, 1.0)
    L.check(L.load().rf_project(ctx.handle, ctypes.byref(g), _ptr(raw5), float(eps), float(delta), _ptr(proj5),
                                _ptr(clip), _stream(stream)), "rf_project")
    return proj5, clip


def rf_project_backward(raw5, clip, eps, delta, dproj5, draw5=None, ctx=None, stream=None):
    """a9: gradients wrt the raw (L, w) from gradients wrt (L, w_proj)."""
    _check_cuda(raw5, torch.float32, name="raw5")
    _check_cuda(dproj5, torch.float32, raw5.shape, name="dproj5")
    _check_cuda(clip, torch.uint8, raw5.shape[1:], name="clip")
    _, ny, nx = raw5.shape
    ctx = ctx or Context.get(raw5.device)
    draw5 = draw5 if draw5 is not None else torch.empty_like(raw5)
    g = _grid(ny, nx, 1.0)
    L.check(L.load().rf_project_backward(ctx.handle, ctypes.byref(g), _ptr(raw5), _ptr(clip), float(eps),
                                         float(delta), _ptr(dproj5), _ptr(draw5), _stream(stream)),
            "rf_project_backward")
    return draw5


def make_opts(tol=0.0, max_sweeps=64, warm=False, band=0, block=0):
    return L.Opts(float(tol), int(max_sweeps), L.RF_MODE_WARM if warm else L.RF_MODE_COLD, int(band), int(block))


def rf_sweep_forward(proj5, eps, src, h, opts=None, T=None, record=True, rec=None, ctx=None, stream=None):
    """a2-a5: forward fast sweep (+ stencil record).  Returns (T, Record|None)."""
    _check_cuda(proj5, torch.float32, name="proj5")
    _, ny, nx = proj5.shape
    _check_cuda(src, torch.uint8, (ny, nx), name="src")
    ctx = ctx or Context.get(proj5.device)
    if T is None:
        T = torch.empty((ny, nx), dtype=torch.float32, device=proj5.device)
    else:
        _check_cuda(T, torch.float32, (ny, nx), name="T")
    if record and rec is None:
        rec = Record.empty(ny, nx, proj5.device)
    o = opts if opts is not None else make_opts()
    g = _grid(ny, nx, h)
    crec = rec.c() if record else None
    L.check(L.load().rf_sweep_forward(ctx.handle, ctypes.byref(g), _ptr(proj5), float(eps), _ptr(src),
                                      ctypes.byref(o), _ptr(T), ctypes.byref(crec) if crec is not None else None,
                                      _stream(stream)), "rf_sweep_forward")
    return T, (rec if record else None)


def rf_record_stencils(proj5, eps, src, h, T, rec=None, ctx=None, stream=None):
    """a5: stencil ids, donor weights and partials of a converged T."""
    _, ny, nx = proj5.shape
    ctx = ctx or Context.get(proj5.device)
    rec = rec if rec is not None else Record.empty(ny, nx, proj5.device)
    g = _grid(ny, nx, h)
    crec = rec.c()
    L.check(L.load().rf_record_stencils(ctx.handle, ctypes.byref(g), _ptr(proj5), float(eps), _ptr(src), _ptr(T),
                                        ctypes.byref(crec), _stream(stream)), "rf_record_stencils")
    return rec


def rf_residual(proj5, eps, src, h, T, per_node=False, ctx=None, stream=None):
    """B7: max |T - min valid candidate(T)| (and the per-node residual)."""
    _, ny, nx = proj5.shape
    ctx = ctx or Context.get(proj5.device)
    res = torch.empty((ny, nx), dtype=torch.float32, device=proj5.device) if per_node else None
    mx = torch.zeros((1,), dtype=torch.float32, device=proj5.device)
    g = _grid(ny, nx, h)
    L.check(L.load().rf_residual(ctx.handle, ctypes.byref(g), _ptr(proj5), float(eps), _ptr(src), _ptr(T),
                                 _ptr(res), _ptr(mx), _stream(stream)), "rf_residual")
    return (mx, res) if per_node else mx


def rf_adjoint(src, T, rec, dLdT, algo="sweep", lam=True, dLdproj5=None, ctx=None, stream=None):
    """a6-a8: solve J^T lambda = g on the recorded stencils and contract with
    the partials.  Returns (dL/d(L11, L21, L22, wx, wy) of the projected
    fields, lambda or None)."""
    ny, nx = T.shape
    _check_cuda(dLdT, torch.float32, (ny, nx), name="dLdT")
    ctx = ctx or Context.get(T.device)
    dLdproj5 = dLdproj5 if dLdproj5 is not None else torch.empty((5, ny, nx), dtype=torch.float32,
                                                                 device=T.device)
    lam_t = torch.empty((ny, nx), dtype=torch.float32, device=T.device) if lam else None
    a = {"sweep": L.RF_ADJ_SWEEP, "ordered": L.RF_ADJ_ORDERED}[algo]
    g = _grid(ny, nx, 1.0)
    crec = rec.c()
    L.check(L.load().rf_adjoint(ctx.handle, ctypes.byref(g), _ptr(src), _ptr(T), ctypes.byref(crec),
                                _ptr(dLdT), _ptr(dLdproj5), _ptr(lam_t), int(a), _stream(stream)), "rf_adjoint")
    return dLdproj5, lam_t
