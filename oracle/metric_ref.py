"""Plain FP64 numpy reference of the paper's learning-side layers (App. B,
"Learning Framework Details: Projections and Regularization").

TEST INFRASTRUCTURE ONLY (imported by tests/ and __graft_entry__.smoke()).
The product path never imports it.

Fields are SoA planes over the grid [ny, nx]:
    gb5 = (g11, g12, g22, b1, b2)   -- the paper's metric G and drift b,
    proj5 = (L11, L21, L22, wx, wy) -- the solver's factor form,
            M = L L^T + eps I = G, w = -b  (sign reading: the solver's cost
            is sqrt(v^T M v) + w^T v and the paper's updates use b = -w).

Forward, following App. B in its order:
  1. eigenvalue clamp of G: lambda_pm = ((g11+g22) +- sqrt((g11-g22)^2 +
     4 g12^2))/2, clamped to [lam_min, lam_max]; principal angle
     theta = atan2(2 g12, g11-g22)/2; G <- U diag(clamped) U^T;
  2. drift: Euclidean norm clipped to b_max ("a safety measure"), then
     n^2 = (b1^2 g22 - 2 b1 b2 g12 + b2^2 g11)/det G with the projected G,
     b <- b (1-delta)/n when n > 1-delta;
  3. (the solver's factor form) L = chol(G - eps I), w = -b.

Backward: the exact derivative of each step, applied in reverse -- for the
clamp the Daleckii-Krein formula for a function of a symmetric matrix
(dF = U (F o (U^T dG U)) U^T with F_ii = f'(lambda_i), F_12 the divided
difference), the quotient rule for the rescalings, and the 2x2 Cholesky
chain.  Component gradients: d/dg12 is the derivative with respect to the
single off-diagonal parameter (it enters G twice).

Total variation (App. B "Total Variation Regularization"), forward
differences D_x f(i,j) = f(i,j+1) - f(i,j) (zero in the last column),
D_y likewise along rows, no grid spacing (the weight absorbs it):
  drift          R(b) = sum_ij sqrt(sum_{d,c} (D_d b_c)^2)
  Frobenius      R(G) = sum_ij sqrt(sum_d (D_d g11)^2 + 2 (D_d g12)^2 + (D_d g22)^2)
  Log-Euclidean  the same with log G (closed form through the same
                 eigendecomposition) in place of G.
Gradients are the subgradient that is 0 where the node's norm is 0.
"""
from __future__ import annotations

import numpy as np


def _a(x):
    return np.asarray(x, np.float64)


# --------------------------------------------------------------------------
# eigendecomposition of a field of symmetric 2x2 matrices (App. B formulas)
# --------------------------------------------------------------------------

def eig2(g11, g12, g22):
    """lambda_+, lambda_-, cos(theta), sin(theta) with the paper's
    trace-discriminant eigenvalues and principal angle
    theta = atan2(2 g12, g11 - g22)/2 (the eigenvector (cos, sin) belongs to
    lambda_+)."""
    g11, g12, g22 = _a(g11), _a(g12), _a(g22)
    r = np.sqrt((g11 - g22) ** 2 + 4.0 * g12 ** 2)
    lp = 0.5 * ((g11 + g22) + r)
    lm = 0.5 * ((g11 + g22) - r)
    th = 0.5 * np.arctan2(2.0 * g12, g11 - g22)
    return lp, lm, np.cos(th), np.sin(th)


def from_eig(mp, mm, c, s):
    """U diag(mp, mm) U^T with U = [[c, -s], [s, c]] -> (o11, o12, o22)."""
    return c * c * mp + s * s * mm, c * s * (mp - mm), s * s * mp + c * c * mm


def _dk_apply(d11, d12, d22, c, s, F11, F12, F22):
    """Daleckii-Krein adjoint on component gradients: S = [[d11, d12/2],
    [d12/2, d22]] -> U (F o (U^T S U)) U^T, returned as components
    (S11, 2 S12, S22)."""
    S11, S12, S22 = d11, 0.5 * d12, d22
    A11 = c * c * S11 + 2 * c * s * S12 + s * s * S22
    A22 = s * s * S11 - 2 * c * s * S12 + c * c * S22
    A12 = -c * s * S11 + (c * c - s * s) * S12 + c * s * S22
    B11, B12, B22 = F11 * A11, F12 * A12, F22 * A22
    o11 = c * c * B11 - 2 * c * s * B12 + s * s * B22
    o22 = s * s * B11 + 2 * c * s * B12 + c * c * B22
    o12 = c * s * B11 + (c * c - s * s) * B12 - c * s * B22
    return o11, 2.0 * o12, o22


# --------------------------------------------------------------------------
# step 1: eigenvalue clamp
# --------------------------------------------------------------------------

def eig_clamp(g11, g12, g22, lam_min, lam_max):
    lp, lm, c, s = eig2(g11, g12, g22)
    return from_eig(np.clip(lp, lam_min, lam_max), np.clip(lm, lam_min, lam_max), c, s)


def eig_clamp_backward(g11, g12, g22, lam_min, lam_max, d11, d12, d22):
    """Gradient of a loss through eig_clamp.  f = clamp: f' = 1 inside
    [lam_min, lam_max] (bounds included), 0 outside; the off-diagonal factor
    is the divided difference (f(l+) - f(l-))/(l+ - l-), f'(l) when l+ = l-."""
    lp, lm, c, s = eig2(g11, g12, g22)
    inside = lambda l: ((l >= lam_min) & (l <= lam_max)).astype(np.float64)
    fp, fm = np.clip(lp, lam_min, lam_max), np.clip(lm, lam_min, lam_max)
    gap = lp - lm
    with np.errstate(divide="ignore", invalid="ignore"):
        F12 = np.where(gap > 0, (fp - fm) / np.where(gap > 0, gap, 1.0), inside(lp))
    return _dk_apply(_a(d11), _a(d12), _a(d22), c, s, inside(lp), F12, inside(lm))


# --------------------------------------------------------------------------
# step 2: drift clip and G^-1-norm rescale
# --------------------------------------------------------------------------

def ginv_norm(b1, b2, g11, g12, g22):
    """|b|_{G^-1} by the closed form of App. B."""
    det = g11 * g22 - g12 * g12
    return np.sqrt((b1 * b1 * g22 - 2 * b1 * b2 * g12 + b2 * b2 * g11) / det)


def drift_project(b1, b2, g11, g12, g22, b_max, c):
    """Euclidean clip to b_max, then rescale to |b|_{G^-1} <= c (c = 1-delta;
    the boundary counts as unclipped)."""
    b1, b2 = _a(b1), _a(b2)
    e = np.hypot(b1, b2)
    se = np.where(e > b_max, b_max / np.where(e > 0, e, 1.0), 1.0)
    e1, e2 = b1 * se, b2 * se
    n = ginv_norm(e1, e2, _a(g11), _a(g12), _a(g22))
    sn = np.where(n > c, c / np.where(n > 0, n, 1.0), 1.0)
    return e1 * sn, e2 * sn


def drift_project_backward(b1, b2, g11, g12, g22, b_max, c, db1, db2):
    """Returns (d b1, d b2, d g11, d g12, d g22) of the raw drift and of the
    (projected) G that the rescale reads."""
    b1, b2, g11, g12, g22 = _a(b1), _a(b2), _a(g11), _a(g12), _a(g22)
    db1, db2 = _a(db1), _a(db2)
    e = np.hypot(b1, b2)
    clip_e = e > b_max
    se = np.where(clip_e, b_max / np.where(e > 0, e, 1.0), 1.0)
    e1, e2 = b1 * se, b2 * se
    det = g11 * g22 - g12 * g12
    p1 = (g22 * e1 - g12 * e2) / det  # G^-1 e
    p2 = (g11 * e2 - g12 * e1) / det
    n2 = e1 * p1 + e2 * p2
    n = np.sqrt(n2)
    clip_n = n > c
    # b_out = c e / n(e, G) where clipped
    bg = db1 * e1 + db2 * e2
    safe_n = np.where(clip_n, n, 1.0)
    de1 = np.where(clip_n, (c / safe_n) * (db1 - p1 * bg / (safe_n * safe_n)), db1)
    de2 = np.where(clip_n, (c / safe_n) * (db2 - p2 * bg / (safe_n * safe_n)), db2)
    # d n / d G = -(G^-1 e)(G^-1 e)^T / (2 n)  ->  dL/dG = c bg/(2 n^3) p p^T
    k = np.where(clip_n, c * bg / (2.0 * safe_n ** 3), 0.0)
    dg11, dg12, dg22 = k * p1 * p1, 2.0 * k * p1 * p2, k * p2 * p2
    # e = b b_max/|b| where clipped
    safe_e = np.where(clip_e, e, 1.0)
    be = b1 * de1 + b2 * de2
    d1 = np.where(clip_e, (b_max / safe_e) * (de1 - b1 * be / (safe_e * safe_e)), de1)
    d2 = np.where(clip_e, (b_max / safe_e) * (de2 - b2 * be / (safe_e * safe_e)), de2)
    return d1, d2, dg11, dg12, dg22


# --------------------------------------------------------------------------
# step 3: the solver's factor form
# --------------------------------------------------------------------------

def chol_eps(g11, g12, g22, eps):
    """L lower-triangular with L L^T = G - eps I."""
    l11 = np.sqrt(_a(g11) - eps)
    l21 = _a(g12) / l11
    l22 = np.sqrt(_a(g22) - eps - l21 * l21)
    return l11, l21, l22


def chol_eps_backward(g11, g12, g22, eps, dl11, dl21, dl22):
    l11, l21, l22 = chol_eps(g11, g12, g22, eps)
    dl11, dl21, dl22 = _a(dl11), _a(dl21), _a(dl22)
    # l22 = sqrt(g22 - eps - l21^2)
    dg22 = dl22 / (2.0 * l22)
    dl21 = dl21 - dl22 * l21 / l22
    # l21 = g12 / l11
    dg12 = dl21 / l11
    dl11 = dl11 - dl21 * l21 / l11
    # l11 = sqrt(g11 - eps)
    dg11 = dl11 / (2.0 * l11)
    return dg11, dg12, dg22


# --------------------------------------------------------------------------
# the composed projection
# --------------------------------------------------------------------------

def metric_project(gb5, lam_min, lam_max, b_max, delta, eps):
    """gb5 (5, ny, nx) raw -> (gbp5 projected (g11, g12, g22, b1, b2),
    proj5 factor form (L11, L21, L22, wx, wy))."""
    g11, g12, g22, b1, b2 = [_a(x) for x in gb5]
    o11, o12, o22 = eig_clamp(g11, g12, g22, lam_min, lam_max)
    p1, p2 = drift_project(b1, b2, o11, o12, o22, b_max, 1.0 - delta)
    l11, l21, l22 = chol_eps(o11, o12, o22, eps)
    return np.stack([o11, o12, o22, p1, p2]), np.stack([l11, l21, l22, -p1, -p2])


def metric_project_backward(gb5, lam_min, lam_max, b_max, delta, eps, dproj5=None, dgbp5=None):
    """Gradient with respect to the raw gb5 of a loss that reads proj5 (with
    gradient dproj5) and/or gbp5 (with gradient dgbp5)."""
    g11, g12, g22, b1, b2 = [_a(x) for x in gb5]
    o11, o12, o22 = eig_clamp(g11, g12, g22, lam_min, lam_max)
    z = np.zeros_like(g11)
    d11 = d12 = d22 = db1 = db2 = z
    if dproj5 is not None:
        dp = [_a(x) for x in dproj5]
        d11, d12, d22 = chol_eps_backward(o11, o12, o22, eps, dp[0], dp[1], dp[2])
        db1, db2 = -dp[3], -dp[4]
    if dgbp5 is not None:
        dq = [_a(x) for x in dgbp5]
        d11, d12, d22 = d11 + dq[0], d12 + dq[1], d22 + dq[2]
        db1, db2 = db1 + dq[3], db2 + dq[4]
    r1, r2, e11, e12, e22 = drift_project_backward(b1, b2, o11, o12, o22, b_max, 1.0 - delta, db1, db2)
    a11, a12, a22 = eig_clamp_backward(g11, g12, g22, lam_min, lam_max, d11 + e11, d12 + e12, d22 + e22)
    return np.stack([a11, a12, a22, r1, r2])


# --------------------------------------------------------------------------
# total variation
# --------------------------------------------------------------------------

def _diffs(f):
    """Forward differences (Dx, Dy) of a [ny, nx] plane, zero on the last
    column / row."""
    dx = np.zeros_like(f)
    dy = np.zeros_like(f)
    dx[:, :-1] = f[:, 1:] - f[:, :-1]
    dy[:-1, :] = f[1:, :] - f[:-1, :]
    return dx, dy


def _diffs_adjoint(ux, uy):
    """Adjoint of _diffs: gradient of sum(ux*Dx f + uy*Dy f) with respect to f."""
    g = np.zeros_like(ux)
    g[:, :-1] -= ux[:, :-1]
    g[:, 1:] += ux[:, :-1]
    g[:-1, :] -= uy[:-1, :]
    g[1:, :] += uy[:-1, :]
    return g


def _tv(planes, weights):
    """sum_ij sqrt(sum_{d,c} w_c (D_d f_c)^2) and its gradient per plane."""
    planes = [_a(p) for p in planes]
    D = [_diffs(p) for p in planes]
    s = sum(w * (dx * dx + dy * dy) for w, (dx, dy) in zip(weights, D))
    N = np.sqrt(s)
    inv = np.where(N > 0, 1.0 / np.where(N > 0, N, 1.0), 0.0)
    grads = [_diffs_adjoint(w * dx * inv, w * dy * inv) for w, (dx, dy) in zip(weights, D)]
    return float(N.sum()), grads


def tv_drift(b1, b2):
    return _tv([b1, b2], [1.0, 1.0])


def tv_frobenius(g11, g12, g22):
    return _tv([g11, g12, g22], [1.0, 2.0, 1.0])


def logm2(g11, g12, g22):
    """Matrix logarithm of an SPD field through the same eigendecomposition."""
    lp, lm, c, s = eig2(g11, g12, g22)
    return from_eig(np.log(lp), np.log(lm), c, s)


def tv_log_euclidean(g11, g12, g22):
    l11, l12, l22 = logm2(g11, g12, g22)
    val, (d11, d12, d22) = _tv([l11, l12, l22], [1.0, 2.0, 1.0])
    # back through log: F_ii = 1/lambda_i, F_12 = (log l+ - log l-)/(l+ - l-)
    lp, lm, c, s = eig2(g11, g12, g22)
    gap = lp - lm
    with np.errstate(divide="ignore", invalid="ignore"):
        F12 = np.where(gap > 0, (np.log(lp) - np.log(lm)) / np.where(gap > 0, gap, 1.0), 1.0 / lp)
    return val, list(_dk_apply(d11, d12, d22, c, s, 1.0 / lp, F12, 1.0 / lm))
