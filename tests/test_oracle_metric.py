"""Pins of the oracle for the paper's learning-side layers (App. B): the
eigenvalue clamp, the drift clip and G^-1-norm rescale, the factor form the
solver reads, and the three total-variation regularisers.  Each forward is
checked against an independent definition (numpy/scipy eigendecomposition,
matrix logarithm, linear solves, closed forms on ramps) and each backward
against central finite differences of its forward."""
import numpy as np
import pytest

from oracle import metric_ref as MR

LMIN, LMAX, BMAX, DELTA, EPS = 0.05, 20.0, 2.0, 0.1, 1e-6


def sym_field(rng, shape, lo=0.2, hi=5.0):
    """Random SPD field with eigenvalues in [lo, hi] and random angles."""
    lp = rng.uniform(lo, hi, shape)
    lm = rng.uniform(lo, hi, shape)
    th = rng.uniform(-np.pi, np.pi, shape)
    c, s = np.cos(th), np.sin(th)
    return c * c * lp + s * s * lm, c * s * (lp - lm), s * s * lp + c * c * lm


def mats(g11, g12, g22):
    return np.stack([np.stack([g11, g12], -1), np.stack([g12, g22], -1)], -2)


def test_eig2_matches_numpy_eigh():
    rng = np.random.default_rng(0)
    g11, g12, g22 = rng.normal(size=(3, 500))
    lp, lm, c, s = MR.eig2(g11, g12, g22)
    w, V = np.linalg.eigh(mats(g11, g12, g22))
    assert np.allclose(lm, w[:, 0], atol=1e-12) and np.allclose(lp, w[:, 1], atol=1e-12)
    # (c, s) is the eigenvector of lambda_+ (up to sign)
    assert np.allclose(np.abs(c * V[:, 0, 1] + s * V[:, 1, 1]), 1.0, atol=1e-10)


def test_eig_clamp_identity_inside_bounds():
    rng = np.random.default_rng(1)
    g = sym_field(rng, (64,), 0.1, 10.0)
    o = MR.eig_clamp(*g, LMIN, LMAX)
    for a, b in zip(o, g):
        assert np.allclose(a, b, atol=1e-13)


def test_eig_clamp_eigenvalues_and_vectors():
    rng = np.random.default_rng(2)
    g11, g12, g22 = rng.normal(scale=10.0, size=(3, 800))  # indefinite and large
    o = MR.eig_clamp(g11, g12, g22, LMIN, LMAX)
    w_in = np.linalg.eigvalsh(mats(g11, g12, g22))
    w_out = np.linalg.eigvalsh(mats(*o))
    assert np.allclose(w_out, np.clip(w_in, LMIN, LMAX), atol=1e-11)
    # same eigenvectors: the output commutes with the input
    A, B = mats(g11, g12, g22), mats(*o)
    assert np.abs(A @ B - B @ A).max() < 1e-9
    # isotropic input (theta = atan2(0, 0)/2 = 0) stays isotropic
    iso = MR.eig_clamp(np.array([0.01, 3.0, 50.0]), np.zeros(3), np.array([0.01, 3.0, 50.0]), LMIN, LMAX)
    assert np.allclose(iso[0], [LMIN, 3.0, LMAX]) and np.allclose(iso[1], 0) and np.allclose(iso[2], iso[0])


def test_ginv_norm_and_drift_projection():
    rng = np.random.default_rng(3)
    g = sym_field(rng, (400,))
    b1, b2 = rng.normal(scale=1.5, size=(2, 400))
    n = MR.ginv_norm(b1, b2, *g)
    A = mats(*g)
    ref = np.sqrt(np.einsum("ni,ni->n", np.stack([b1, b2], -1), np.linalg.solve(A, np.stack([b1, b2], -1)[..., None])[..., 0]))
    assert np.allclose(n, ref, rtol=1e-12)
    c = 1.0 - DELTA
    p1, p2 = MR.drift_project(b1, b2, *g, BMAX, c)
    e = np.hypot(b1, b2)
    ne = ref * np.minimum(1.0, BMAX / e)  # norm after the Euclidean clip
    assert np.allclose(MR.ginv_norm(p1, p2, *g), np.minimum(ne, c), rtol=1e-12)
    assert np.all(np.hypot(p1, p2) <= BMAX * (1 + 1e-12))
    # direction preserved
    assert np.allclose(p1 * b2 - p2 * b1, 0.0, atol=1e-12) and np.all(p1 * b1 + p2 * b2 >= 0)
    # feasible drift is untouched
    q1, q2 = MR.drift_project(0.01 * b1, 0.01 * b2, *g, BMAX, c)
    assert np.allclose(q1, 0.01 * b1) and np.allclose(q2, 0.01 * b2)


def test_cholesky_factor_form():
    rng = np.random.default_rng(4)
    g = sym_field(rng, (300,))
    l11, l21, l22 = MR.chol_eps(*g, EPS)
    L = np.zeros((300, 2, 2))
    L[:, 0, 0], L[:, 1, 0], L[:, 1, 1] = l11, l21, l22
    assert np.allclose(L @ np.swapaxes(L, 1, 2) + EPS * np.eye(2), mats(*g), atol=1e-12)
    gb = np.stack([*g, *rng.normal(size=(2, 300))])
    gbp, proj = MR.metric_project(gb, LMIN, LMAX, BMAX, DELTA, EPS)
    assert np.allclose(proj[3], -gbp[3]) and np.allclose(proj[4], -gbp[4])


def fd(f, xs, i, h=1e-6):
    """Central difference of scalar f with respect to xs[i] (all entries)."""
    out = np.zeros_like(xs[i])
    for k in np.ndindex(xs[i].shape):
        xp = [x.copy() for x in xs]
        xm = [x.copy() for x in xs]
        xp[i][k] += h
        xm[i][k] -= h
        out[k] = (f(*xp) - f(*xm)) / (2 * h)
    return out


def clamp_cases(rng, n):
    """Matrices whose eigenvalues sit inside, below and above the bounds,
    away from the kinks by a margin."""
    lp = rng.choice([0.01, 0.03, 1.0, 3.0, 30.0, 60.0], n) * rng.uniform(0.9, 1.1, n)
    lm = rng.choice([0.01, 0.03, 0.5, 2.0, 40.0], n) * rng.uniform(0.9, 1.1, n)
    th = rng.uniform(-np.pi, np.pi, n)
    c, s = np.cos(th), np.sin(th)
    return c * c * lp + s * s * lm, c * s * (lp - lm), s * s * lp + c * c * lm


def test_eig_clamp_backward_matches_finite_differences():
    rng = np.random.default_rng(5)
    g = [x.copy() for x in clamp_cases(rng, 24)]
    w = rng.normal(size=(3, 24))
    loss = lambda a, b, c: float(sum((wi * oi).sum() for wi, oi in zip(w, MR.eig_clamp(a, b, c, LMIN, LMAX))))
    got = MR.eig_clamp_backward(*g, LMIN, LMAX, *w)
    for i in range(3):
        assert np.allclose(got[i], fd(loss, g, i), atol=1e-6, rtol=1e-6), i


def test_drift_project_backward_matches_finite_differences():
    rng = np.random.default_rng(6)
    n = 30
    g = list(sym_field(rng, (n,)))
    b = list(rng.normal(scale=1.2, size=(2, n)))
    b[0][:5] *= 5.0  # some Euclidean clips
    w = rng.normal(size=(2, n))
    c = 1.0 - DELTA
    loss = lambda b1, b2, g11, g12, g22: float(sum((wi * oi).sum() for wi, oi in zip(w, MR.drift_project(b1, b2, g11, g12, g22, BMAX, c))))
    xs = [b[0], b[1], *g]
    got = MR.drift_project_backward(*xs, BMAX, c, *w)
    e = np.hypot(*b)
    assert (e > BMAX).any() and (MR.ginv_norm(*MR.drift_project(*b, *g, BMAX, 1e9), *g) > c).any()
    for i in range(5):
        assert np.allclose(got[i], fd(loss, xs, i), atol=1e-6, rtol=1e-6), i


def test_metric_project_backward_matches_finite_differences():
    rng = np.random.default_rng(7)
    n = 20
    g = clamp_cases(rng, n)
    gb = np.stack([*g, *rng.normal(scale=1.0, size=(2, n))])
    wp, wq = rng.normal(size=(2, 5, n))
    def loss(*planes):
        gbp, proj = MR.metric_project(np.stack(planes), LMIN, LMAX, BMAX, DELTA, EPS)
        return float((wp * proj).sum() + (wq * gbp).sum())
    got = MR.metric_project_backward(gb, LMIN, LMAX, BMAX, DELTA, EPS, dproj5=wp, dgbp5=wq)
    xs = [p.copy() for p in gb]
    for i in range(5):
        assert np.allclose(got[i], fd(loss, xs, i), atol=2e-6, rtol=1e-5), i


def test_tv_closed_forms_on_ramps():
    ny, nx, a, c = 7, 9, 0.3, -0.7
    J, I = np.meshgrid(np.arange(nx, dtype=float), np.arange(ny, dtype=float))
    z = np.zeros((ny, nx))
    # Frobenius: diagonal ramp a per step; the off-diagonal counts twice
    assert np.isclose(MR.tv_frobenius(a * J, z, z)[0], abs(a) * (nx - 1) * ny)
    assert np.isclose(MR.tv_frobenius(z, a * J, z)[0], np.sqrt(2) * abs(a) * (nx - 1) * ny)
    assert np.isclose(MR.tv_frobenius(z, z, c * I)[0], abs(c) * nx * (ny - 1))
    # drift: coupled norm; interior sqrt(a^2+c^2), last column |c|, last row |a|
    want = (nx - 1) * (ny - 1) * np.hypot(a, c) + (ny - 1) * abs(c) + (nx - 1) * abs(a)
    assert np.isclose(MR.tv_drift(a * J, c * I)[0], want)
    # Log-Euclidean: G = exp(a j) I -> log G = a j I, norm sqrt(2)|a|
    e = np.exp(a * J)
    assert np.isclose(MR.tv_log_euclidean(e, z, e)[0], np.sqrt(2) * abs(a) * (nx - 1) * ny)


def test_tv_rotation_invariance_and_logm():
    scipy_linalg = pytest.importorskip("scipy.linalg")
    rng = np.random.default_rng(8)
    g = sym_field(rng, (6, 8))
    th = 0.7
    R = np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
    Gr = R @ mats(*g) @ R.T
    gr = (Gr[..., 0, 0], Gr[..., 0, 1], Gr[..., 1, 1])
    assert np.isclose(MR.tv_log_euclidean(*g)[0], MR.tv_log_euclidean(*gr)[0], rtol=1e-12)
    assert np.isclose(MR.tv_frobenius(*g)[0], MR.tv_frobenius(*gr)[0], rtol=1e-12)
    l11, l12, l22 = MR.logm2(*g)
    A = mats(*g)
    for k in [(0, 0), (2, 5), (5, 7)]:
        Lref = scipy_linalg.logm(A[k]).real
        assert np.allclose([l11[k], l12[k], l22[k]], [Lref[0, 0], Lref[0, 1], Lref[1, 1]], atol=1e-12)


@pytest.mark.parametrize("which", ["drift", "frobenius", "log_euclidean"])
def test_tv_gradients_match_finite_differences(which):
    rng = np.random.default_rng(9)
    g = [x.copy() for x in sym_field(rng, (5, 6))]
    if which == "drift":
        xs = [x.copy() for x in rng.normal(size=(2, 5, 6))]
        f = MR.tv_drift
    elif which == "frobenius":
        xs, f = g, MR.tv_frobenius
    else:
        xs, f = g, MR.tv_log_euclidean
    _, grads = f(*xs)
    for i in range(len(xs)):
        assert np.allclose(grads[i], fd(lambda *p: f(*p)[0], xs, i), atol=1e-6, rtol=1e-6), i
