"""The paper's forward-solver validation suite (App. "Forward Solver
Validation"; Table 1; the iteration table of the same appendix) and its
pointwise gradient verification (Sec. 4.2 table of gradient accuracy; App.
"Gradient Verification"), as regression tests of the FP64 oracle against
the values the paper prints (fixture tests/golden/validation_appendix.txt,
which also states the readings)."""
import math
import os

import numpy as np
import pytest

import oracle as O
from oracle import metric_ref as MR

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "validation_appendix.txt")


def golden():
    out = {}
    for line in open(GOLDEN):
        line = line.split("#")[0].strip()
        if line:
            k, v, _ = line.split()
            out[k] = float(v)
    return out


def rot(l1, l2, th):
    c, s = math.cos(th), math.sin(th)
    R = np.array([[c, -s], [s, c]])
    return R @ np.diag([l1, l2]) @ R.T


def raw_from_g(g11, g12, g22, b1, b2):
    """Factor form (L, w) of the paper's (G, b): M = L L^T = G, w = -b."""
    l11, l21, l22 = MR.chol_eps(g11, g12, g22, 0.0)
    return np.stack([l11, l21, l22, -np.asarray(b1, float), -np.asarray(b2, float)]).astype(np.float64)


def full(n, v):
    return np.full((n, n), float(v))


def solve(n, G=None, b=(0.0, 0.0), srcs=None, fields=None):
    """Oracle GS solve on N x N nodes, h = 1/N, source(s) (row, col)."""
    h = 1.0 / n
    if fields is None:
        fields = (full(n, G[0, 0]), full(n, G[0, 1]), full(n, G[1, 1]), full(n, b[0]), full(n, b[1]))
    raw = raw_from_g(*fields)
    srcs = srcs or [(n // 2, n // 2)]
    src = np.zeros((n, n), np.uint8)
    for i, j in srcs:
        src[i, j] = 1
    proj, _ = O.project(raw, 0.0, 0.05)
    T, iters, st, _ = O.solve_gs(proj, src, h, 0.0)
    assert st == O.OK
    return T, iters, h, src


def exact(n, h, G, b, srcs):
    y, x = np.mgrid[0:n, 0:n] * h
    best = np.full((n, n), np.inf)
    for i, j in srcs:
        dx, dy = x - j * h, y - i * h
        best = np.minimum(best, np.sqrt(G[0, 0] * dx * dx + 2 * G[0, 1] * dx * dy + G[1, 1] * dy * dy)
                          - b[0] * dx - b[1] * dy)
    return best


def rel_l2(T, E):
    return 100.0 * float(np.sqrt(np.mean((T - E) ** 2)) / E.max())


def max_pointwise(T, E):
    return 100.0 * float(np.abs(T - E).max() / E.max())


def close(got, want, tol):
    return abs(got - want) <= tol * abs(want)


def test_table1_relative_column():
    g = golden()
    for n in (25, 50, 100, 200, 400):
        T, _, h, _ = solve(n, np.eye(2))
        c = n // 2
        E = exact(n, h, np.eye(2), (0, 0), [(c, c)])
        assert close(rel_l2(T, E), g[f"table1_rel_l2_{n}"], 0.15 if n == 25 else 0.07), n


def test_anisotropic_and_rotated_metrics():
    g = golden()
    n = 200
    c = n // 2
    G = np.diag([4.0, 0.25])
    T, _, h, _ = solve(n, G)
    E = exact(n, h, G, (0, 0), [(c, c)])
    assert close(rel_l2(T, E), g["diag_rel_l2_200"], 0.10)
    assert close(max_pointwise(T, E), g["diag_max_pointwise_200"], 0.10)
    G = rot(4.0, 0.25, math.pi / 4)
    assert abs(G[0, 1] - 1.875) < 1e-12
    T, _, h, _ = solve(n, G)
    assert close(rel_l2(T, exact(n, h, G, (0, 0), [(c, c)])), g["rotated_rel_l2_200"], 0.10)


def test_combined_randers_richardson():
    g = golden()
    G, b = rot(2.0, 0.5, math.pi / 6), (0.2, 0.1)
    T1, _, _, _ = solve(100, G, b)
    T4, _, _, _ = solve(400, G, b)
    fine = T4[::4, ::4]
    d = 100.0 * np.linalg.norm(T1 - fine) / np.linalg.norm(fine)
    assert close(d, g["combined_richardson"], 0.25), d


def test_piecewise_media_slowdown():
    g = golden()
    n = 200
    j = np.arange(n)[None, :] * np.ones((n, 1))
    gg = np.where(j < n // 2, 1.0, 4.0)
    z = np.zeros((n, n))
    T, _, h, _ = solve(n, fields=(gg, z, gg, z, z), srcs=[(n // 2, n // 4)])
    row = T[n // 2]
    fast = (row[n // 4 + 20] - row[n // 4 + 5]) / (15 * h)
    slow = (row[n - 10] - row[n - 40]) / (30 * h)
    assert close(slow / fast, g["piecewise_slowdown"], 0.01)


def test_smooth_media_eikonal_residual():
    g = golden()
    n = 200
    j = np.arange(n)[None, :] * np.ones((n, 1))
    gg = 1.0 + 0.5 * np.sin(2 * np.pi * j / n)
    z = np.zeros((n, n))
    T, _, h, _ = solve(n, fields=(gg, z, gg, z, z))
    ty, tx = np.gradient(T, h)
    res = np.abs(np.hypot(tx, ty) / np.sqrt(gg) - 1.0)
    yy, xx = np.mgrid[0:n, 0:n]
    m = np.hypot(yy - n // 2, xx - n // 2) > 5
    m[0, :] = m[-1, :] = m[:, 0] = m[:, -1] = False
    assert close(100.0 * res[m].mean(), g["smooth_mean_residual_200"], 0.15)


def test_multiple_ignition_points():
    g = golden()
    n = 200
    srcs = [(n // 4, n // 4), (n // 4, 3 * n // 4), (3 * n // 4, n // 2)]
    T, _, h, _ = solve(n, np.eye(2), srcs=srcs)
    assert close(rel_l2(T, exact(n, h, np.eye(2), (0, 0), srcs)), g["multisource_rel_l2_200"], 0.10)


def test_iterations_independent_of_size():
    g = golden()
    for n in (50, 100, 200, 400):
        _, iters, _, _ = solve(n, np.eye(2))
        assert iters == g["iterations"], (n, iters)


# ---- pointwise gradient verification ----------------------------------------

def loss_and_grad(fields, src, h, obs, That):
    """L = 1/2 sum_obs (T - T^)^2 and dL/d(g11, g12, g22, b1, b2) by the
    oracle's adjoint (Alg. 2) chained through the factor form."""
    raw = raw_from_g(*fields)
    proj, clip = O.project(raw, 0.0, 0.05)
    assert not clip.any()
    T, _, st, _ = O.solve_gs(proj, src, h, 0.0)
    assert st == O.OK
    gT = np.where(obs, T - That, 0.0)
    rec = O.record(proj, src, h, 0.0, T)
    _, gproj = O.adjoint(src, T, rec, gT)
    d11, d12, d22 = MR.chol_eps_backward(fields[0], fields[1], fields[2], 0.0, gproj[0], gproj[1], gproj[2])
    return 0.5 * float((gT * gT).sum()), np.stack([d11, d12, d22, -gproj[3], -gproj[4]]), rec


def loss_only(fields, src, h, obs, That):
    proj, _ = O.project(raw_from_g(*fields), 0.0, 0.05)
    T, _, st, _ = O.solve_gs(proj, src, h, 0.0)
    assert st == O.OK
    d = np.where(obs, T - That, 0.0)
    return 0.5 * float((d * d).sum())


GRAD_CASES = {
    "isotropic": ((np.eye(2), (0.0, 0.0)), [0, 1, 2, 3, 4]),
    "anisotropic": ((rot(2.0, 0.5, math.pi / 6), (0.0, 0.0)), [0, 1, 2]),
    "drift": ((np.eye(2), (0.15, 0.08)), [3, 4]),
}


def gradient_case(name, n=40, points=20, seed=0):
    (G, b), comps = GRAD_CASES[name]
    h = 1.0 / n
    fields = [full(n, G[0, 0]), full(n, G[0, 1]), full(n, G[1, 1]), full(n, b[0]), full(n, b[1])]
    src = np.zeros((n, n), np.uint8)
    src[n // 2, n // 2] = 1
    rng = np.random.default_rng(seed)
    obs = rng.random((n, n)) < 0.3  # MSE on 30 % of the cells (Sec. 4 backward workload)
    proj, _ = O.project(raw_from_g(*fields), 0.0, 0.05)
    T0, _, _, _ = O.solve_gs(proj, src, h, 0.0)
    That = 0.9 * T0
    L0, grad, rec = loss_and_grad(fields, src, h, obs, That)
    tmax = T0.max()
    cand = [(i, j) for i in range(3, n - 3) for j in range(3, n - 3)
            if max(abs(i - n // 2), abs(j - n // 2)) > 2 and rec["margin"][i, j] > 1e-4 * tmax]
    pick = [cand[k] for k in rng.choice(len(cand), size=points, replace=False)]
    return fields, src, h, obs, That, grad, pick, comps


@pytest.mark.parametrize("name", list(GRAD_CASES))
def test_pointwise_gradients_match_finite_differences(name):
    """Central differences with the paper's step 1e-5 at 20 random interior
    points agree with the implicit gradient to a relative 1e-6 (the paper's
    bound), for the isotropic, anisotropic and drift configurations."""
    fields, src, h, obs, That, grad, pick, comps = gradient_case(name)
    eps = 1e-5
    scale = np.abs(grad[comps]).max()
    for (i, j) in pick:
        for c in comps:
            fp = [f.copy() for f in fields]
            fm = [f.copy() for f in fields]
            fp[c][i, j] += eps
            fm[c][i, j] -= eps
            fd = (loss_only(fp, src, h, obs, That) - loss_only(fm, src, h, obs, That)) / (2 * eps)
            den = max(abs(fd), 1e-3 * scale)
            assert abs(grad[c, i, j] - fd) <= 1e-6 * den, (name, (i, j), c, grad[c, i, j], fd)


@pytest.mark.parametrize("name", ["isotropic", "anisotropic"])
def test_gradient_stability_under_metric_noise(name):
    """1 % metric noise moves the mean gradient by well under 1 % (the paper
    reports 0.48 %; the reading of the measure is in the fixture)."""
    g = golden()
    n = 40
    fields, src, h, obs, That, grad, _, _ = gradient_case(name, n=n)
    var = []
    for k in range(10):
        r = np.random.default_rng(100 + k)
        f2 = [f.copy() for f in fields]
        f2[0] = f2[0] * (1 + 0.01 * r.standard_normal((n, n)))
        f2[2] = f2[2] * (1 + 0.01 * r.standard_normal((n, n)))
        _, g2, _ = loss_and_grad(f2, src, h, obs, That)
        m0, m1 = grad[:3].mean(axis=(1, 2)), g2[:3].mean(axis=(1, 2))
        var.append(np.abs(m1 - m0).sum() / np.abs(m0).sum())
    assert 100.0 * np.mean(var) < 2.0 * g["stability_mean_gradient_variation"], np.mean(var)


@pytest.mark.parametrize("name", ["isotropic", "anisotropic"])
def test_random_direction_derivatives(name):
    """Directional derivatives along 100 random unit directions of the whole
    parameter space (all five fields at every node): the implicit gradient
    matches central differences wherever the perturbation keeps every
    node's active stencil, and with the exactly converged FP64 solve no
    direction switches a stencil at step 1e-5 here (the paper's 20 %
    success rate comes from directions that cross stencil boundaries)."""
    n = 40
    fields, src, h, obs, That, grad, _, _ = gradient_case(name, n=n)
    proj, _ = O.project(raw_from_g(*fields), 0.0, 0.05)
    T0, _, _, _ = O.solve_gs(proj, src, h, 0.0)
    ids0 = O.record(proj, src, h, 0.0, T0)["id"]
    eps = 1e-5
    kept = 0
    for k in range(100):
        v = np.random.default_rng(1000 + k).standard_normal((5, n, n))
        v /= np.linalg.norm(v)
        fp = [f + eps * v[c] for c, f in enumerate(fields)]
        fm = [f - eps * v[c] for c, f in enumerate(fields)]
        pp, _ = O.project(raw_from_g(*fp), 0.0, 0.05)
        Tp, _, _, _ = O.solve_gs(pp, src, h, 0.0)
        if (O.record(pp, src, h, 0.0, Tp)["id"] != ids0).any():
            continue
        kept += 1
        fd = (loss_only(fp, src, h, obs, That) - loss_only(fm, src, h, obs, That)) / (2 * eps)
        assert abs(fd - float((grad * v).sum())) <= 1e-5 * abs(fd), (k, fd)
    assert kept >= 90
