"""The paper's validation suite through the CUDA path (the oracle-side
version and the readings are in tests/test_oracle_validation.py and
tests/golden/validation_appendix.txt): forward errors against the printed
values, sweep counts, and the pointwise gradients of the paper's (G, b)
parameterisation against FP64 central differences."""
import math

import numpy as np
import pytest

import oracle as O
from gpu_util import FWD_TOL, require_gpu, to_dev, torch
from paper_2603_00035_gb300 import api
from paper_2603_00035_gb300.autograd import metric_solve
from test_oracle_validation import (close, exact, full, golden, gradient_case, loss_only, max_pointwise,
                                    raw_from_g, rel_l2, rot)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def gpu_solve(n, G=None, b=(0.0, 0.0), srcs=None, fields=None, variant=0):
    h = 1.0 / n
    if fields is None:
        fields = (full(n, G[0, 0]), full(n, G[0, 1]), full(n, G[1, 1]), full(n, b[0]), full(n, b[1]))
    raw = raw_from_g(*fields).astype(np.float32)
    srcs = srcs or [(n // 2, n // 2)]
    src = np.zeros((n, n), np.uint8)
    for i, j in srcs:
        src[i, j] = 1
    proj, _ = api.rf_project(to_dev(raw), 0.0, 0.05)
    T, _ = api.rf_sweep_forward(proj, 0.0, to_dev(src, torch.uint8), h, opts=api.make_opts(variant=variant),
                                record=False)
    st = api.Context.get(0).stats()
    assert st["status"] == 0 and st["converged"], st
    # reference: the oracle on the same float32-rounded fields
    prj, _ = O.project(raw.astype(np.float64), 0.0, 0.05)
    To, _, _, _ = O.solve_gs(prj, src, h, 0.0)
    Tg = T.cpu().numpy().astype(np.float64)
    assert np.abs(Tg - To).max() <= FWD_TOL * To.max()
    return Tg, st["sweeps"], h


@pytest.mark.parametrize("variant", ["streamed", "tiled1"])
def test_forward_validation_suite_on_gpu(variant):
    g = golden()
    n = 200
    c = n // 2
    G = np.diag([4.0, 0.25])
    T, sweeps, h = gpu_solve(n, G, variant=variant)
    E = exact(n, h, G, (0, 0), [(c, c)])
    assert close(rel_l2(T, E), g["diag_rel_l2_200"], 0.10)
    assert close(max_pointwise(T, E), g["diag_max_pointwise_200"], 0.10)
    G = rot(4.0, 0.25, math.pi / 4)
    T, _, h = gpu_solve(n, G, variant=variant)
    assert close(rel_l2(T, exact(n, h, G, (0, 0), [(c, c)])), g["rotated_rel_l2_200"], 0.10)
    srcs = [(n // 4, n // 4), (n // 4, 3 * n // 4), (3 * n // 4, n // 2)]
    T, _, h = gpu_solve(n, np.eye(2), srcs=srcs, variant=variant)
    assert close(rel_l2(T, exact(n, h, np.eye(2), (0, 0), srcs)), g["multisource_rel_l2_200"], 0.10)
    G, b = rot(2.0, 0.5, math.pi / 6), (0.2, 0.1)
    T1, _, _ = gpu_solve(100, G, b, variant=variant)
    T4, _, _ = gpu_solve(400, G, b, variant=variant)
    d = 100.0 * np.linalg.norm(T1 - T4[::4, ::4]) / np.linalg.norm(T4[::4, ::4])
    assert close(d, g["combined_richardson"], 0.25)
    j = np.arange(n)[None, :] * np.ones((n, 1))
    gg = 1.0 + 0.5 * np.sin(2 * np.pi * j / n)
    z = np.zeros((n, n))
    T, _, h = gpu_solve(n, fields=(gg, z, gg, z, z), variant=variant)
    ty, tx = np.gradient(T, h)
    res = np.abs(np.hypot(tx, ty) / np.sqrt(gg) - 1.0)
    yy, xx = np.mgrid[0:n, 0:n]
    m = np.hypot(yy - c, xx - c) > 5
    m[0, :] = m[-1, :] = m[:, 0] = m[:, -1] = False
    assert close(100.0 * res[m].mean(), g["smooth_mean_residual_200"], 0.15)


def test_sweep_count_independent_of_size():
    """The paper's solver converges in 2 iterations (4 sweeps each) at every
    size; the GPU's line sweeps (the paper's schedule), which stop at the
    first sweep that changes nothing, need at most one more iteration to
    prove it."""
    g = golden()
    for n in (50, 100, 200, 400, 800):
        _, sweeps, _ = gpu_solve(n, np.eye(2), variant="streamed")
        assert sweeps <= 4 * (g["iterations"] + 1), (n, sweeps)


@pytest.mark.parametrize("name", ["isotropic", "anisotropic", "drift"])
def test_pointwise_gradients_on_gpu(name):
    """The CUDA path's gradient of the paper's (G, b) parameters (App. B
    projection with non-binding bounds -> solve -> adjoint -> projection
    backward) against FP64 central differences of the oracle at the same 20
    interior points, to FP32 accuracy."""
    fields, src, h, obs, That, _, pick, comps = gradient_case(name)
    prm = api.metric_params(1e-3, 1e3, 1e3, 0.05, 0.0)
    x = to_dev(np.stack(fields).astype(np.float32)).requires_grad_(True)
    T, _ = metric_solve(x, to_dev(src, torch.uint8), h, prm)
    obs_t, That_t = to_dev(obs.astype(np.float32)), to_dev(That.astype(np.float32))
    loss = 0.5 * (obs_t * (T - That_t) ** 2).sum()
    loss.backward()
    assert api.Context.get(0).stats()["status"] == 0
    gg = x.grad.cpu().numpy().astype(np.float64)
    eps = 1e-5
    fds = {}
    for (i, j) in pick:
        for c in comps:
            fp = [f.copy() for f in fields]
            fm = [f.copy() for f in fields]
            fp[c][i, j] += eps
            fm[c][i, j] -= eps
            fds[(i, j, c)] = (loss_only(fp, src, h, obs, That) - loss_only(fm, src, h, obs, That)) / (2 * eps)
    scale = max(abs(v) for v in fds.values())
    for (i, j, c), fd in fds.items():
        assert abs(gg[c, i, j] - fd) <= 1e-3 * max(abs(fd), 1e-2 * scale), (name, (i, j), c, gg[c, i, j], fd)
