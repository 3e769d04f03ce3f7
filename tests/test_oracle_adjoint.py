"""Pins of the oracle's backward pass (Alg. 2, Eqs. 4-7) and projection.

* mass conservation: donor weights sum to one, so the multipliers that reach
  the sources add up to the total loss gradient;
* Euler identity: T is positively homogeneous of degree one in (L, w) when
  eps = 0, so sum_theta theta dL/dtheta = sum_i g_i T_i;
* the reverse-order back-substitution equals a sparse direct solve of
  (I - W^T) lambda = g (scipy's spsolve);
* central finite differences of the full solve on random parameters away
  from stencil switches (paper: relative error < 1e-6);
* projection: feasible drifts unchanged, clipped drifts land on the
  |w|_{M^-1} = 1 - delta sphere, backward equals finite differences.
"""
import numpy as np
import pytest
from scipy.sparse import coo_matrix, identity
from scipy.sparse.linalg import spsolve

import oracle as O
import rf_inputs as R

DX = [-1, -1, -1, 0, 1, 1, 1, 0]
DY = [1, 0, -1, -1, -1, 0, 1, 1]


def small_case(seed=0, ny=48, nx=44, eps=0.0, omega_scale=0.3):
    h = 1.0 / (max(ny, nx) - 1)
    raw = R.randers_fields(ny, nx, h, 8, seed, omega="unit", omega_scale=omega_scale)
    src = R.random_sources(ny, nx, 2, seed, margin=3)
    g = R.sparse_loss_grad(ny, nx, 0.2, seed)
    return raw.astype(np.float64), src, h, eps, g.astype(np.float64)


def test_mass_conservation_and_euler_identity():
    raw, src, h, eps, g = small_case()
    out = O.solve_and_grad(raw, src, h, eps, 0.05, g)
    assert out["status"] == O.OK
    assert not out["clip"].any()
    lam = out["lam"]
    assert lam[src == 1].sum() == pytest.approx(g.sum(), rel=1e-10)
    euler = (raw * out["graw"]).sum()
    assert euler == pytest.approx((g * out["T"]).sum(), rel=1e-10)


def test_back_substitution_matches_sparse_solve():
    raw, src, h, eps, g = small_case(seed=4, ny=30, nx=27)
    out = O.solve_and_grad(raw, src, h, eps, 0.05, g)
    rec, T = out["rec"], out["T"]
    ny, nx = T.shape
    ids, jac = rec["id"], rec["jac"]
    rows, cols, vals = [], [], []
    for i in range(ny):
        for j in range(nx):
            q = i * nx + j
            a = int(ids[i, j])
            if a == 0:
                continue
            kind, k = a >> 4, a & 7
            donors = [k] if kind == 1 else [k, (k + 1) % 8]
            for slot, n in enumerate(donors):
                p = (i + DY[n]) * nx + (j + DX[n])
                # W[q, p] = dT_q / dT_p = -J_qp / J_qq
                rows.append(q)
                cols.append(p)
                vals.append(-jac[1 + slot, i, j] / jac[0, i, j])
    W = coo_matrix((vals, (rows, cols)), shape=(ny * nx, ny * nx)).tocsc()
    lam = spsolve((identity(ny * nx, format="csc") - W.T).tocsc(), g.ravel())
    assert np.allclose(out["lam"].ravel(), lam, rtol=1e-10, atol=1e-12)
    # the weights of every active update are a convex combination
    s = np.zeros(ny * nx)
    np.add.at(s, rows, vals)
    active = ids.ravel() != 0
    assert np.allclose(s[active], 1.0, atol=1e-12)
    assert min(vals) >= -1e-15


def loss(raw, src, h, eps, delta, g):
    proj, _ = O.project(raw, eps, delta)
    T, _, st, _ = O.solve_gs(proj, src, h, eps)
    rec = O.record(proj, src, h, eps, T)
    return float((g * T).sum()), rec["id"]


@pytest.mark.parametrize("seed,delta,omega", [(0, 0.05, 0.3), (2, 0.5, 0.6)])
def test_finite_differences(seed, delta, omega):
    raw, src, h, eps, g = small_case(seed=seed, ny=40, nx=36, eps=1e-6, omega_scale=omega)
    out = O.solve_and_grad(raw, src, h, eps, delta, g)
    if delta == 0.5:
        assert out["clip"].any()  # the clip branch is exercised
    rng = np.random.default_rng(seed)
    ny, nx = src.shape
    checked = 0
    for t in range(32):
        c = int(rng.integers(0, 5))
        i, j = int(rng.integers(0, ny)), int(rng.integers(0, nx))
        if src[i, j]:
            continue
        e = 1e-6 * max(1.0, abs(raw[c, i, j]))
        rp = raw.copy()
        rp[c, i, j] += e
        rm = raw.copy()
        rm[c, i, j] -= e
        lp, idp = loss(rp, src, h, eps, delta, g)
        lm, idm = loss(rm, src, h, eps, delta, g)
        if not np.array_equal(idp, idm) or not np.array_equal(idp, out["rec"]["id"]):
            continue  # a stencil switch inside the FD interval
        fd = (lp - lm) / (2 * e)
        an = out["graw"][c, i, j]
        assert an == pytest.approx(fd, rel=1e-5, abs=1e-8 * max(1.0, np.abs(g).sum()))
        checked += 1
    assert checked >= 20


def test_projection_closed_form_cases():
    rng = np.random.default_rng(0)
    n = 200
    raw = np.zeros((5, n))
    th = rng.uniform(0, np.pi, n)
    a = rng.uniform(0.5, 2, n)
    b = rng.uniform(0.5, 2, n)
    l11, l21, l22 = R.metric_factor(th, a, b, 0.0)
    raw[0], raw[1], raw[2] = l11, l21, l22
    raw[3], raw[4] = rng.uniform(-2, 2, n), rng.uniform(-2, 2, n)
    eps, delta = 1e-3, 0.25
    proj, clip = O.project(raw, eps, delta)
    for p in range(n):
        L = np.array([[raw[0, p], 0], [raw[1, p], raw[2, p]]])
        M = L @ L.T + eps * np.eye(2)
        w = raw[3:, p]
        nrm = np.sqrt(w @ np.linalg.solve(M, w))
        wp = proj[3:, p]
        assert np.allclose(proj[:3, p], raw[:3, p])
        if nrm <= 1 - delta:
            assert not clip[p] and np.allclose(wp, w, rtol=0, atol=0)
        else:
            assert clip[p]
            assert np.sqrt(wp @ np.linalg.solve(M, wp)) == pytest.approx(1 - delta, rel=1e-12)
            assert abs(wp[0] * w[1] - wp[1] * w[0]) < 1e-12 and wp @ w > 0  # same direction
    assert 20 < clip.sum() < n - 20


def test_projection_backward_finite_differences():
    rng = np.random.default_rng(1)
    n = 64
    raw = np.zeros((5, n))
    l11, l21, l22 = R.metric_factor(rng.uniform(0, np.pi, n), rng.uniform(0.5, 2, n), rng.uniform(0.5, 2, n), 0.0)
    raw[0], raw[1], raw[2] = l11, l21, l22
    raw[3], raw[4] = rng.uniform(-1.5, 1.5, n), rng.uniform(-1.5, 1.5, n)
    eps, delta = 1e-2, 0.3
    gproj = rng.standard_normal((5, n))
    _, clip = O.project(raw, eps, delta)
    graw = O.project_backward(raw, clip, eps, delta, gproj)
    f = lambda r: float((O.project(r, eps, delta)[0] * gproj).sum())
    for c in range(5):
        for p in range(n):
            e = 1e-6
            rp = raw.copy()
            rp[c, p] += e
            rm = raw.copy()
            rm[c, p] -= e
            _, cp = O.project(rp, eps, delta)
            _, cm = O.project(rm, eps, delta)
            if cp[p] != cm[p]:
                continue
            fd = (f(rp) - f(rm)) / (2 * e)
            assert graw[c, p] == pytest.approx(fd, rel=1e-6, abs=1e-8)
