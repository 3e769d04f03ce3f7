"""FP64 CPU oracle for the differentiable Randers eikonal solver.

TEST INFRASTRUCTURE ONLY: ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product path (``paper_2603_00035_gb300``) never imports it.

The arithmetic lives in ``rf_oracle.c`` (plain C, double precision), compiled
by :func:`build` with gcc into ``liborc.so`` beside it.  This module only
marshals numpy arrays to it.  Every function cites the paper passage it
follows; see the C file for the equations.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rf_oracle.c")
_LIB = os.path.join(_HERE, "liborc.so")

OK, ERR_INVALID_ARG, ERR_NOT_CONVERGED, ERR_NO_SOURCE = 0, 1, 3, 6

_lib = None


def build(force: bool = False) -> str:
    """Compile rf_oracle.c into liborc.so (gcc, -O2, no arch flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", _SRC, "-o", _LIB, "-lm"]
        subprocess.run(cmd, check=True)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        I, I64, D = ctypes.c_int, ctypes.c_int64, ctypes.c_double
        lib.orc_cell_eval.argtypes = [P, D, D, D, D, D, D, P, P, P, P, P]
        lib.orc_cell_eval.restype = None
        lib.orc_project.argtypes = [I64, P, P, P, P, P, D, D, P, P, P]
        lib.orc_project_backward.argtypes = [I64, P, P, P, P, P, P, D, D, P, P]
        lib.orc_solve_gs.argtypes = [I, I, D, D, P, P, P, P, P, P, P, I, I, P, P]
        lib.orc_solve_ordered.argtypes = [I, I, D, D, P, P, P, P, P, P, P]
        lib.orc_residual.argtypes = [I, I, D, D, P, P, P, P, P, P, P, P]
        lib.orc_record.argtypes = [I, I, D, D, P, P, P, P, P, P, P, P, P, P, P, P]
        lib.orc_adjoint.argtypes = [I, I, P, P, P, P, P, P, P, P]
        lib.orc_cell_softmin.argtypes = [P, D, D, D, D, D, D, D, P, P]
        lib.orc_cell_softmin.restype = D
        lib.orc_solve_softmin_gs.argtypes = [I, I, D, D, P, P, P, P, P, P, D, D, I, P, P]
        lib.orc_softmin_record.argtypes = [I, I, D, D, P, P, P, P, P, P, P, D, P, P]
        lib.orc_softmin_adjoint.argtypes = [I, I, P, P, P, P, P, D, I, P, P, P]
        for f in ("orc_project", "orc_project_backward", "orc_solve_gs", "orc_solve_ordered",
                  "orc_residual", "orc_record", "orc_adjoint", "orc_solve_softmin_gs", "orc_softmin_record",
                  "orc_softmin_adjoint"):
            getattr(lib, f).restype = ctypes.c_int
        _lib = lib
    return _lib


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _u8(a):
    return np.ascontiguousarray(a, dtype=np.uint8)


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def cell_eval(Tn, h, g11, g12, g22, wx, wy):
    """Candidates of one node from its eight neighbour times (Eqs. 2-3, App. A).

    Returns dict with two-point candidates/validity/lambda per stencil and
    one-point candidates/validity per neighbour.
    """
    lib = _load()
    Tn = _d(Tn)
    two = np.zeros(8)
    two_ok = np.zeros(8, np.int32)
    lam = np.zeros(16)
    one = np.zeros(8)
    one_ok = np.zeros(8, np.int32)
    lib.orc_cell_eval(_p(Tn), h, g11, g12, g22, wx, wy, _p(two), _p(two_ok), _p(lam), _p(one), _p(one_ok))
    return dict(two=two, two_ok=two_ok.astype(bool), lam=lam.reshape(8, 2), one=one,
                one_ok=one_ok.astype(bool))


def project(raw5, eps, delta):
    """Feasibility projection (App. B; metric in factor form M = L L^T + eps I).

    raw5: array (5, ...) of L11, L21, L22, wx, wy.  Returns (proj5, clip)
    where proj5 = (L11, L21, L22, wpx, wpy).
    """
    lib = _load()
    raw5 = _d(raw5)
    shape = raw5.shape[1:]
    n = int(np.prod(shape))
    r = raw5.reshape(5, n)
    wpx, wpy = np.zeros(n), np.zeros(n)
    clip = np.zeros(n, np.uint8)
    st = lib.orc_project(n, _p(r[0]), _p(r[1]), _p(r[2]), _p(r[3]), _p(r[4]), eps, delta,
                         _p(wpx), _p(wpy), _p(clip))
    if st != OK:
        raise ValueError(f"orc_project status {st}")
    proj = np.stack([r[0], r[1], r[2], wpx, wpy]).reshape((5,) + shape)
    return proj, clip.reshape(shape)


def project_backward(raw5, clip, eps, delta, gproj5):
    """Backward of :func:`project`: gradients wrt raw (L, w) from gradients
    wrt (L, w_proj)."""
    lib = _load()
    raw5 = _d(raw5)
    shape = raw5.shape[1:]
    n = int(np.prod(shape))
    r = raw5.reshape(5, n)
    gin = _d(gproj5).reshape(5 * n)
    gout = np.zeros(5 * n)
    clip = _u8(clip).reshape(n)
    st = lib.orc_project_backward(n, _p(r[0]), _p(r[1]), _p(r[2]), _p(r[3]), _p(r[4]), _p(clip),
                                  eps, delta, _p(gin), _p(gout))
    if st != OK:
        raise ValueError(f"orc_project_backward status {st}")
    return gout.reshape((5,) + shape)


def _fields(proj5):
    f = _d(proj5)
    return f, [f[c] for c in range(5)]


def solve_gs(proj5, src, h, eps, max_iter=200, replace=True):
    """Gauss-Seidel fast sweeping (Alg. 1).  Returns (T, iterations, status, updates)."""
    lib = _load()
    f, (l11, l21, l22, wx, wy) = _fields(proj5)
    ny, nx = f.shape[1:]
    src = _u8(src)
    T = np.zeros((ny, nx))
    it = ctypes.c_int(0)
    upd = ctypes.c_int64(0)
    st = lib.orc_solve_gs(ny, nx, h, eps, _p(l11), _p(l21), _p(l22), _p(wx), _p(wy), _p(src), _p(T),
                          max_iter, int(replace), ctypes.byref(it), ctypes.byref(upd))
    return T, it.value, st, upd.value


def solve_ordered(proj5, src, h, eps):
    """Ordered (label-setting) solve of the same discrete system."""
    lib = _load()
    f, (l11, l21, l22, wx, wy) = _fields(proj5)
    ny, nx = f.shape[1:]
    src = _u8(src)
    T = np.zeros((ny, nx))
    st = lib.orc_solve_ordered(ny, nx, h, eps, _p(l11), _p(l21), _p(l22), _p(wx), _p(wy), _p(src), _p(T))
    return T, st


def residual(proj5, src, h, eps, T):
    """r = T - min valid candidate(T) at every non-source node."""
    lib = _load()
    f, (l11, l21, l22, wx, wy) = _fields(proj5)
    ny, nx = f.shape[1:]
    T = _d(T)
    src = _u8(src)
    res = np.zeros((ny, nx))
    lib.orc_residual(ny, nx, h, eps, _p(l11), _p(l21), _p(l22), _p(wx), _p(wy), _p(src), _p(T), _p(res))
    return res


def record(proj5, src, h, eps, T):
    """Stencil identification and residual partials (Alg. 2 first loop, App. A).

    Returns dict: id (uint8), jac (3, ny, nx) = dR/d(T0, donor1, donor2),
    drt (5, ny, nx) = dR/d(L11, L21, L22, wx, wy), margin (second - best),
    geo_only (count of causality-rejected geometric-valid two-point
    candidates), and the derived normalised quantities w1 = -J_1/J_0 (donor
    weight) and dT (5, ny, nx) = -dR/dtheta / dR/dT0.
    """
    lib = _load()
    f, (l11, l21, l22, wx, wy) = _fields(proj5)
    ny, nx = f.shape[1:]
    T = _d(T)
    src = _u8(src)
    n = ny * nx
    ids = np.zeros((ny, nx), np.uint8)
    jac = np.zeros((3, ny, nx))
    drt = np.zeros((5, ny, nx))
    margin = np.zeros((ny, nx))
    geo = ctypes.c_int64(0)
    lib.orc_record(ny, nx, h, eps, _p(l11), _p(l21), _p(l22), _p(wx), _p(wy), _p(src), _p(T), _p(ids),
                   _p(jac), _p(drt), _p(margin), ctypes.byref(geo))
    active = ids != 0
    j0 = np.where(active, jac[0], 1.0)
    w1 = np.where(active, -jac[1] / j0, 0.0)
    dT = np.where(active[None], -drt / j0[None], 0.0)
    del n
    return dict(id=ids, jac=jac, drt=drt, margin=margin, geo_only=geo.value, w1=w1, dT=dT)


def adjoint(src, T, rec, g):
    """Reverse-T back-substitution and parameter gradients (Alg. 2; Eqs. 4-6).

    Returns (lam_norm, grad5) with lam_norm the unit-diagonal multiplier and
    grad5 = dL/d(L11, L21, L22, w_proj x, w_proj y).
    """
    lib = _load()
    T = _d(T)
    ny, nx = T.shape
    src = _u8(src)
    g = _d(g)
    lam = np.zeros((ny, nx))
    grad = np.zeros((5, ny, nx))
    ids = _u8(rec["id"])
    jac = _d(rec["jac"])
    drt = _d(rec["drt"])
    st = lib.orc_adjoint(ny, nx, _p(src), _p(T), _p(ids), _p(jac), _p(drt), _p(g), _p(lam), _p(grad))
    if st != OK:
        raise ValueError(f"orc_adjoint status {st}")
    return lam, grad


def solve_and_grad(raw5, src, h, eps, delta, g, max_iter=200):
    """Whole path on the CPU: project -> GS solve -> record -> adjoint ->
    project backward.  Returns dict with every intermediate."""
    proj, clip = project(raw5, eps, delta)
    T, iters, st, upd = solve_gs(proj, src, h, eps, max_iter)
    rec = record(proj, src, h, eps, T)
    g = np.where(np.isfinite(T), g, 0.0)
    lam, gproj = adjoint(src, T, rec, g)
    graw = project_backward(raw5, clip, eps, delta, gproj)
    return dict(proj=proj, clip=clip, T=T, iters=iters, status=st, updates=upd, rec=rec, lam=lam,
                gproj=gproj, graw=graw)


# ---- soft-min relaxation (Sec. 3.3 names it; the formula is this build's reading) ----

def cell_softmin(Tn, h, g11, g12, g22, wx, wy, tau):
    """Soft-min of one node over its 8 stencil values (each the minimum of
    its segment: the valid two-point candidate, else the smaller endpoint
    one-point candidate): (T0, p[8] softmax weights of the stencils,
    from[8] the candidate behind each value: 8 + k two-point of stencil k, n
    one-point through neighbour n, -1 none)."""
    lib = _load()
    p = np.zeros(8)
    frm = np.zeros(8, np.int32)
    T0 = lib.orc_cell_softmin(_p(_d(Tn)), h, g11, g12, g22, wx, wy, tau, _p(p), _p(frm))
    return T0, p, frm


def solve_softmin(proj5, src, h, eps, tau, tol=1e-14, max_iter=2000):
    """Gauss-Seidel sweeps of T = softmin_tau(candidates(T)).  Returns (T,
    iterations, status)."""
    lib = _load()
    f, (l11, l21, l22, wx, wy) = _fields(proj5)
    ny, nx = f.shape[1:]
    src = _u8(src)
    T = np.zeros((ny, nx))
    it = ctypes.c_int(0)
    st = lib.orc_solve_softmin_gs(ny, nx, h, eps, _p(l11), _p(l21), _p(l22), _p(wx), _p(wy), _p(src), tau, tol,
                                  max_iter, _p(T), ctypes.byref(it))
    return T, it.value, st


def softmin_record(proj5, src, h, eps, T, tau):
    """(wnb (8, ny, nx) = dT/dT(neighbour n), dth (5, ny, nx) = dT/dtheta)."""
    lib = _load()
    f, (l11, l21, l22, wx, wy) = _fields(proj5)
    ny, nx = f.shape[1:]
    wnb = np.zeros((8, ny, nx))
    dth = np.zeros((5, ny, nx))
    lib.orc_softmin_record(ny, nx, h, eps, _p(l11), _p(l21), _p(l22), _p(wx), _p(wy), _p(_u8(src)), _p(_d(T)), tau,
                           _p(wnb), _p(dth))
    return wnb, dth


def softmin_adjoint(src, T, wnb, dth, g, tol=1e-15, max_pass=200):
    """(lambda, grad5, passes) of the soft-min system."""
    lib = _load()
    T = _d(T)
    ny, nx = T.shape
    lam = np.zeros((ny, nx))
    grad = np.zeros((5, ny, nx))
    passes = ctypes.c_int(0)
    st = lib.orc_softmin_adjoint(ny, nx, _p(_u8(src)), _p(T), _p(_d(wnb)), _p(_d(dth)), _p(_d(g)), tol, max_pass,
                                 _p(lam), _p(grad), ctypes.byref(passes))
    if st != OK:
        raise ValueError(f"orc_softmin_adjoint status {st}")
    return lam, grad, passes.value


def softmin_solve_and_grad(raw5, src, h, eps, delta, g, tau):
    """Whole soft-min path on the CPU: project -> soft solve -> record ->
    adjoint -> project backward."""
    proj, clip = project(raw5, eps, delta)
    T, iters, st = solve_softmin(proj, src, h, eps, tau)
    wnb, dth = softmin_record(proj, src, h, eps, T, tau)
    g = np.where(np.isfinite(T), g, 0.0)
    lam, gproj, passes = softmin_adjoint(src, T, wnb, dth, g)
    graw = project_backward(raw5, clip, eps, delta, gproj)
    return dict(proj=proj, clip=clip, T=T, iters=iters, status=st, wnb=wnb, dth=dth, lam=lam, gproj=gproj, graw=graw,
                passes=passes)
