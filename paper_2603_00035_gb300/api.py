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

    def set_adjoint_park(self, ns: int):
        """RF_ADJ_TILES: stall (ns) before a waiting tile yields its CTA."""
        L.check(L.load().rf_ctx_set_adjoint_park(self.handle, int(ns)), "rf_ctx_set_adjoint_park")

    def raise_on_device_error(self, where: str):
        """Synchronise the last call's stream and raise RFError when the
        device status word holds an error (RF_ERR_NOT_CONVERGED,
        RF_ERR_TIMEOUT, RF_ERR_NONFINITE_INPUT, RF_ERR_NO_SOURCE ...).  The
        word is cleared by the read, so each error is reported once."""
        st = self.stats()
        if st["status"] != L.RF_OK:
            raise L.RFError(st["status"], where)
        return st

    def stats(self) -> dict:
        st = L.Stats()
        L.load().rf_ctx_last_stats(self.handle, ctypes.byref(st))
        return dict(status=st.status, status_name=L.STATUS.get(st.status, str(st.status)), sweeps=st.sweeps,
                    converged=bool(st.converged), adj_sweeps=st.adj_sweeps, cell_updates=st.cell_updates,
                    max_residual=st.max_residual, rounds=st.rounds)

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


def metric_params(lam_min=1e-2, lam_max=1e2, b_max=None, delta=0.05, eps=1e-6):
    """rf_metric_params of App. B's projection: eigenvalues clamped to
    [lam_min, lam_max], |b|_2 <= b_max (default (1-delta) sqrt(lam_max), the
    largest Euclidean norm a feasible drift can have), |b|_{G^-1} <= 1-delta;
    eps is the solver's (M = L L^T + eps I)."""
    if b_max is None:
        b_max = (1.0 - delta) * lam_max ** 0.5
    return L.MetricParams(float(lam_min), float(lam_max), float(b_max), float(delta), float(eps))


def rf_metric_project(gb5, prm, gbp5=None, proj5=None, want_gbp=True, want_proj=True, ctx=None, stream=None):
    """App. B projection of the paper's (g11, g12, g22, b1, b2): returns
    (gbp5 projected, proj5 the solver's factor form); either may be skipped.
    gbp5 may be gb5 itself (in-place projection)."""
    _check_cuda(gb5, torch.float32, name="gb5")
    _, ny, nx = gb5.shape
    ctx = ctx or Context.get(gb5.device)
    if want_gbp and gbp5 is None:
        gbp5 = torch.empty_like(gb5)
    if want_proj and proj5 is None:
        proj5 = torch.empty_like(gb5)
    g = _grid(ny, nx, 1.0)
    L.check(L.load().rf_metric_project(ctx.handle, ctypes.byref(g), _ptr(gb5), ctypes.byref(prm),
                                       _ptr(gbp5) if want_gbp else None, _ptr(proj5) if want_proj else None,
                                       _stream(stream)), "rf_metric_project")
    return (gbp5 if want_gbp else None), (proj5 if want_proj else None)


def rf_metric_project_backward(gb5, prm, dproj5=None, dgbp5=None, dgb5=None, ctx=None, stream=None):
    """Gradient wrt the raw gb5 from gradients wrt proj5 and/or gbp5."""
    _check_cuda(gb5, torch.float32, name="gb5")
    for t, nm in ((dproj5, "dproj5"), (dgbp5, "dgbp5")):
        if t is not None:
            _check_cuda(t, torch.float32, gb5.shape, name=nm)
    _, ny, nx = gb5.shape
    ctx = ctx or Context.get(gb5.device)
    dgb5 = dgb5 if dgb5 is not None else torch.empty_like(gb5)
    g = _grid(ny, nx, 1.0)
    L.check(L.load().rf_metric_project_backward(ctx.handle, ctypes.byref(g), _ptr(gb5), ctypes.byref(prm),
                                                _ptr(dproj5), _ptr(dgbp5), _ptr(dgb5), _stream(stream)),
            "rf_metric_project_backward")
    return dgb5


TV_METRIC = {"none": L.RF_TV_NONE, "frobenius": L.RF_TV_FROBENIUS, "log_euclidean": L.RF_TV_LOG_EUCLIDEAN}


def rf_tv(gb5, metric="frobenius", w_metric=1.0, w_drift=1.0, grad5=None, value=True, ctx=None, stream=None):
    """App. B total variation of (G, b): returns (values [R(G), R(b)] as a
    CUDA float32 tensor or None, grad5) with grad5 += w_metric dR(G) +
    w_drift dR(b) when grad5 is given."""
    _check_cuda(gb5, torch.float32, name="gb5")
    if grad5 is not None:
        _check_cuda(grad5, torch.float32, gb5.shape, name="grad5")
    _, ny, nx = gb5.shape
    ctx = ctx or Context.get(gb5.device)
    mode = TV_METRIC[metric] if isinstance(metric, str) else int(metric)
    val = torch.empty(2, dtype=torch.float32, device=gb5.device) if value else None
    g = _grid(ny, nx, 1.0)
    L.check(L.load().rf_tv(ctx.handle, ctypes.byref(g), _ptr(gb5), mode, float(w_metric), float(w_drift),
                           _ptr(val), _ptr(grad5), _stream(stream)), "rf_tv")
    return val, grad5


SWEEP_VARIANTS = {"auto": L.RF_SWEEP_AUTO, "tiled1": L.RF_SWEEP_TILED1, "streamed": L.RF_SWEEP_STREAMED,
                  "tiled4": L.RF_SWEEP_TILED4, "tiles": L.RF_SWEEP_TILES}

# adjoint schedules (enum rf_adjoint_algo); "ordered", "levels" and "tiles"
# give the same multipliers and gradients bit for bit
ADJ_ALGOS = {"sweep": L.RF_ADJ_SWEEP, "ordered": L.RF_ADJ_ORDERED, "levels": L.RF_ADJ_LEVELS,
             "tiles": L.RF_ADJ_TILES}


def make_opts(tol=0.0, max_sweeps=64, warm=False, band=0, block=0, rtol=1e-6, variant=0, window=0.0):
    """rf_opts: a node counts as changed when |dT| > tol + rtol * T (tol =
    rtol = 0: bitwise); the solve stops at a state where no node changes.
    band/block: line-tile shape of the line-sweep variants (0 = auto);
    variant: forward kernel, a name of SWEEP_VARIANTS or its value (0 =
    auto); window: the tile queue's delta-stepping window in tile crossings
    (0 = auto)."""
    v = SWEEP_VARIANTS[variant] if isinstance(variant, str) else int(variant)
    return L.Opts(float(tol), int(max_sweeps), L.RF_MODE_WARM if warm else L.RF_MODE_COLD, int(band), int(block),
                  float(rtol), v, float(window))


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


def rf_adjoint(src, T, rec, dLdT, algo="tiles", lam=True, dLdproj5=None, ctx=None, stream=None):
    """a6-a8: solve J^T lambda = g on the recorded stencils and contract with
    the partials.  algo: a name of ADJ_ALGOS.  Returns (dL/d(L11,
    L21, L22, wx, wy) of the projected fields, lambda or None)."""
    ny, nx = T.shape
    _check_cuda(dLdT, torch.float32, (ny, nx), name="dLdT")
    ctx = ctx or Context.get(T.device)
    dLdproj5 = dLdproj5 if dLdproj5 is not None else torch.empty((5, ny, nx), dtype=torch.float32,
                                                                 device=T.device)
    lam_t = torch.empty((ny, nx), dtype=torch.float32, device=T.device) if lam else None
    a = ADJ_ALGOS[algo]
    g = _grid(ny, nx, 1.0)
    crec = rec.c()
    L.check(L.load().rf_adjoint(ctx.handle, ctypes.byref(g), _ptr(src), _ptr(T), ctypes.byref(crec),
                                _ptr(dLdT), _ptr(dLdproj5), _ptr(lam_t), int(a), _stream(stream)), "rf_adjoint")
    return dLdproj5, lam_t


def rf_step_host(raw5_h, src_h, dLdT_h, h, eps, delta, T_h, dLdraw_h, opts=None, algo="tiles", ctx=None,
                 stream=None, device=0):
    """Whole steps (project, solve, record, adjoint, project back) on host
    tensors, pipelined across steps inside the library: lists of CPU tensors
    (preferably pinned) raw5_h [5, ny, nx] float32, src_h [ny, nx] uint8,
    dLdT_h [ny, nx] float32, and outputs T_h [ny, nx], dLdraw_h [5, ny, nx]
    float32, one entry per step.  Returns when the outputs are filled."""
    nsteps = len(raw5_h)
    if not (len(src_h) == len(dLdT_h) == len(T_h) == len(dLdraw_h) == nsteps):
        raise ValueError("one input and output set per step")
    _, ny, nx = raw5_h[0].shape if nsteps else (5, 1, 1)
    for t, dt, shp in [(x, torch.float32, (5, ny, nx)) for x in raw5_h] + [(x, torch.uint8, (ny, nx)) for x in src_h] + \
            [(x, torch.float32, (ny, nx)) for x in dLdT_h] + [(x, torch.float32, (ny, nx)) for x in T_h] + \
            [(x, torch.float32, (5, ny, nx)) for x in dLdraw_h]:
        if t.is_cuda or t.dtype != dt or tuple(t.shape) != shp or not t.is_contiguous():
            raise ValueError(f"host tensor {dt} {shp} contiguous expected, got {t.dtype} {tuple(t.shape)}")
    ctx = ctx or Context.get(torch.device("cuda", device))
    arr = lambda ts: (ctypes.c_void_p * max(1, nsteps))(*[t.data_ptr() for t in ts])
    o = opts if opts is not None else make_opts()
    a = ADJ_ALGOS[algo]
    g = _grid(ny, nx, h)
    L.check(L.load().rf_step_host(ctx.handle, ctypes.byref(g), nsteps, arr(raw5_h), arr(src_h), arr(dLdT_h),
                                  float(eps), float(delta), ctypes.byref(o), int(a), arr(T_h), arr(dLdraw_h),
                                  _stream(stream)), "rf_step_host")


# ---- soft-min relaxation (Sec. 3.3) -----------------------------------------------

def rf_softmin_forward(proj5, eps, src, h, tau, opts=None, T=None, ctx=None, stream=None):
    """Relaxed forward solve: T = softmin_tau over the 8 stencil values."""
    _check_cuda(proj5, torch.float32, name="proj5")
    _, ny, nx = proj5.shape
    _check_cuda(src, torch.uint8, (ny, nx), name="src")
    ctx = ctx or Context.get(proj5.device)
    T = T if T is not None else torch.empty((ny, nx), dtype=torch.float32, device=proj5.device)
    o = opts if opts is not None else make_opts()
    g = _grid(ny, nx, h)
    L.check(L.load().rf_softmin_forward(ctx.handle, ctypes.byref(g), _ptr(proj5), float(eps), _ptr(src), float(tau),
                                        ctypes.byref(o), _ptr(T), _stream(stream)), "rf_softmin_forward")
    return T


def rf_softmin_record(proj5, eps, src, h, T, tau, ctx=None, stream=None):
    """(wnb (8, ny, nx), dT (5, ny, nx)) of the relaxed system at T."""
    _, ny, nx = proj5.shape
    ctx = ctx or Context.get(proj5.device)
    wnb = torch.empty((8, ny, nx), dtype=torch.float32, device=proj5.device)
    dT = torch.empty((5, ny, nx), dtype=torch.float32, device=proj5.device)
    g = _grid(ny, nx, h)
    L.check(L.load().rf_softmin_record(ctx.handle, ctypes.byref(g), _ptr(proj5), float(eps), _ptr(src), _ptr(T),
                                       float(tau), _ptr(wnb), _ptr(dT), _stream(stream)), "rf_softmin_record")
    return wnb, dT


def rf_softmin_adjoint(src, T, wnb, dT, dLdT, lam=True, dLdproj5=None, ctx=None, stream=None):
    """(dL/d(L11, L21, L22, wx, wy), lambda or None) of the relaxed system."""
    ny, nx = T.shape
    _check_cuda(dLdT, torch.float32, (ny, nx), name="dLdT")
    ctx = ctx or Context.get(T.device)
    dLdproj5 = dLdproj5 if dLdproj5 is not None else torch.empty((5, ny, nx), dtype=torch.float32, device=T.device)
    lam_t = torch.empty((ny, nx), dtype=torch.float32, device=T.device) if lam else None
    g = _grid(ny, nx, 1.0)
    L.check(L.load().rf_softmin_adjoint(ctx.handle, ctypes.byref(g), _ptr(src), _ptr(T), _ptr(wnb), _ptr(dT),
                                        _ptr(dLdT), _ptr(dLdproj5), _ptr(lam_t), _stream(stream)),
            "rf_softmin_adjoint")
    return dLdproj5, lam_t


# ---- a10: batched solve ------------------------------------------------------

BATCH_DESC_DTYPE = None  # numpy structured dtype matching rf_batch_desc


def _desc_dtype():
    import numpy as np
    global BATCH_DESC_DTYPE
    if BATCH_DESC_DTYPE is None:
        BATCH_DESC_DTYPE = np.dtype([("ny", "<i4"), ("nx", "<i4"), ("h", "<f4"), ("pad", "<i4"), ("offset", "<i8")])
        assert BATCH_DESC_DTYPE.itemsize == ctypes.sizeof(L.BatchDesc)
    return BATCH_DESC_DTYPE


class BatchSolver:
    """Packs many grids into the layout rf_batch_solve expects and runs the
    forward (+ adjoint) of all of them in one persistent launch; optionally
    captured once in a CUDA graph and replayed.

    grids: list of dicts with raw (5, ny, nx) float32, src (ny, nx) uint8,
    h, and optionally g (ny, nx) float32 (dL/dT).  Grids are stored largest
    first; `order[k]` is the caller's index of packed grid k.
    """

    def __init__(self, grids, eps=1e-6, delta=0.05, device="cuda", opts=None, ctx=None):
        import numpy as np
        dev = torch.device(device)
        self.eps, self.delta = float(eps), float(delta)
        self.ctx = ctx or Context.get(dev)
        self.opts = opts if opts is not None else make_opts()
        sizes = [g["src"].size for g in grids]
        self.order = sorted(range(len(grids)), key=lambda k: -sizes[k])
        self.n = len(grids)
        offs, off = [], 0
        for k in self.order:
            offs.append(off)
            off += int(grids[k]["src"].size)
        self.total = off
        self.max_line = max(max(g["src"].shape) for g in grids)
        desc = np.zeros(self.n, dtype=_desc_dtype())
        raw = np.zeros((5, self.total), np.float32)
        src = np.zeros(self.total, np.uint8)
        has_g = all("g" in g for g in grids)
        gg = np.zeros(self.total, np.float32) if has_g else None
        for slot, k in enumerate(self.order):
            g = grids[k]
            ny, nx = g["src"].shape
            o = offs[slot]
            desc[slot] = (ny, nx, g["h"], 0, o)
            raw[:, o:o + ny * nx] = g["raw"].reshape(5, -1)
            src[o:o + ny * nx] = g["src"].reshape(-1)
            if has_g:
                gg[o:o + ny * nx] = g["g"].reshape(-1)
        self.offsets = offs
        self.shapes = [grids[k]["src"].shape for k in self.order]
        self.desc = torch.from_numpy(desc.view(np.uint8)).to(dev)
        self.raw = torch.from_numpy(raw).to(dev)
        self.src = torch.from_numpy(src).to(dev)
        self.g = torch.from_numpy(gg).to(dev) if has_g else None
        self.proj = torch.empty_like(self.raw)
        self.clip = torch.empty(self.total, dtype=torch.uint8, device=dev)
        self.T = torch.empty(self.total, dtype=torch.float32, device=dev)
        self.rec = Record(torch.empty(self.total, dtype=torch.uint8, device=dev),
                          torch.empty(self.total, dtype=torch.float32, device=dev),
                          torch.empty((5, self.total), dtype=torch.float32, device=dev))
        self.gproj = torch.empty_like(self.raw) if has_g else None
        self.graw = torch.empty_like(self.raw) if has_g else None
        self.gstat = torch.zeros((self.n, 3), dtype=torch.int32, device=dev)
        self.graph = None

    def _launch(self, stream=None):
        flat = L.Grid(1, int(self.total), 1.0)
        lib = L.load()
        st = _stream(stream)
        L.check(lib.rf_project(self.ctx.handle, ctypes.byref(flat), _ptr(self.raw), self.eps, self.delta,
                               _ptr(self.proj), _ptr(self.clip), st), "rf_project")
        crec = self.rec.c()
        L.check(lib.rf_batch_solve(self.ctx.handle, _ptr(self.desc), int(self.n), int(self.total),
                                   int(self.max_line), _ptr(self.proj), self.eps, _ptr(self.src),
                                   ctypes.byref(self.opts), _ptr(self.T), ctypes.byref(crec), _ptr(self.g),
                                   _ptr(self.gproj), _ptr(self.gstat), st), "rf_batch_solve")
        if self.g is not None:
            L.check(lib.rf_project_backward(self.ctx.handle, ctypes.byref(flat), _ptr(self.raw), _ptr(self.clip),
                                            self.eps, self.delta, _ptr(self.gproj), _ptr(self.graw), st),
                    "rf_project_backward")

    def run(self):
        """Project, solve every grid (and its adjoint), project backward."""
        if self.graph is not None:
            self.graph.replay()
        else:
            self._launch()

    def capture(self):
        """Capture one run in a CUDA graph (after a warm-up run that sizes
        the workspace); later run() calls replay it."""
        self._launch()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            with torch.cuda.graph(g, stream=s):
                self._launch(stream=s)
        torch.cuda.current_stream().wait_stream(s)
        self.graph = g
        return g

    def grid(self, k, what="T"):
        """Result of the caller's grid k: T (ny, nx), graw (5, ny, nx), the
        record fields (id, w1) or the per-grid status."""
        slot = self.order.index(k)
        o = self.offsets[slot]
        ny, nx = self.shapes[slot]
        if what == "T":
            return self.T[o:o + ny * nx].view(ny, nx)
        if what == "graw":
            return self.graw[:, o:o + ny * nx].reshape(5, ny, nx)
        if what == "id":
            return self.rec.id[o:o + ny * nx].view(ny, nx)
        if what == "w1":
            return self.rec.w1[o:o + ny * nx].view(ny, nx)
        if what == "status":
            return self.gstat[slot]
        raise ValueError(what)
