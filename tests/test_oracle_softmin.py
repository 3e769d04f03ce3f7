"""Pins of the FP64 oracle's soft-min relaxation (Sec. 3.3 names soft-min
stencil selection; the formula is this build's reading: T0 = -tau log
sum_k exp(-c_k/tau) over the 8 stencil values c_k, each the minimum of its
segment -- the valid two-point candidate, else the smaller one-point
candidate of its endpoints):

* the local soft-min equals a logsumexp (scipy) of stencil values built from
  the hard update's own candidates (orc_cell_eval), with softmax weights;
* it is continuous where a two-point candidate turns valid (lambda = 0);
* tau -> 0 recovers the hard solution (orc_solve_gs) and its record;
* the relaxed solution lies below the hard one and decreases with tau, and
  every node lies within tau log(#candidates) below its candidate minimum;
* the record's weights sum to 1 per node, so the adjoint conserves mass
  (sum of the source multipliers = sum of g);
* the adjoint gradient matches central finite differences of the FP64 soft
  solve on random parameters, and across a stencil switch where the hard
  solution has a kink.
"""
import numpy as np
import pytest

import oracle as O
import rf_inputs as R

scipy_special = pytest.importorskip("scipy.special")


def setup(n=24, seed=3, K=4):
    h = 1.0 / (n - 1)
    raw = R.randers_fields(n, n, h, K, seed=seed, omega="unit", omega_scale=0.3).astype(np.float64)
    src = R.random_sources(n, n, 2, seed=seed)
    prj, _ = O.project(raw, 1e-6, 0.05)
    return raw, src, prj, h


def _random_node(rng):
    Tn = rng.uniform(0.0, 1.0, 8)
    Tn[rng.random(8) < 0.3] = np.inf
    a, b, th = rng.uniform(0.5, 2.0), rng.uniform(0.5, 2.0), rng.uniform(0, np.pi)
    Rm = np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
    M = Rm @ np.diag([a * a, b * b]) @ Rm.T
    w = rng.uniform(-0.2, 0.2, 2)
    return Tn, M, w


def test_local_softmin_is_logsumexp_of_the_stencil_values():
    rng = np.random.default_rng(0)
    for trial in range(300):
        Tn, M, w = _random_node(rng)
        h, tau = 0.05, rng.uniform(1e-3, 2e-2)
        c = O.cell_eval(Tn, h, M[0, 0], M[0, 1], M[1, 1], w[0], w[1])
        one = np.where(c["one_ok"], c["one"], np.inf)
        vals = np.array([c["two"][k] if c["two_ok"][k] else min(one[k], one[(k + 1) % 8]) for k in range(8)])
        T0, p, frm = O.cell_softmin(Tn, h, M[0, 0], M[0, 1], M[1, 1], w[0], w[1], tau)
        fin = np.isfinite(vals)
        if not fin.any():
            assert np.isinf(T0) and not p.any() and (frm == -1).all()
            continue
        want = -tau * scipy_special.logsumexp(-vals[fin] / tau)
        assert T0 == pytest.approx(want, rel=1e-12, abs=1e-12)
        assert np.allclose(p[fin], scipy_special.softmax(-vals[fin] / tau), rtol=1e-10, atol=1e-14)
        assert not p[~fin].any()
        assert np.min(vals[fin]) - tau * np.log(fin.sum()) - 1e-12 <= T0 <= np.min(vals[fin]) + 1e-12
        # tau = 0: the hard minimum over all valid candidates
        T00, _, _ = O.cell_softmin(Tn, h, M[0, 0], M[0, 1], M[1, 1], w[0], w[1], 0.0)
        allv = np.concatenate([np.where(c["two_ok"], c["two"], np.inf), one])
        assert T00 == np.min(allv)


def test_local_softmin_is_continuous_where_a_two_point_turns_valid():
    """Move one donor time across the point where a stencil's two-point
    candidate becomes valid (a barycentric weight crosses 0): the soft value
    changes by O(step), not by a jump."""
    h, tau = 0.05, 2e-3
    M = np.eye(2)
    base = np.full(8, np.inf)
    base[1] = 0.30  # neighbour 1 (-1, 0); stencil 0 pairs neighbours 0 and 1
    # scan neighbour 0's time: the two-point candidate of stencil 0 switches
    ts = np.linspace(0.30, 0.40, 20001)
    vals, valid = [], []
    for t in ts:
        Tn = base.copy()
        Tn[0] = t
        T0, p, frm = O.cell_softmin(Tn, h, 1.0, 0.0, 1.0, 0.0, 0.0, tau)
        vals.append(T0)
        valid.append(frm[0] == 8)
    vals, valid = np.array(vals), np.array(valid)
    assert valid.any() and (~valid).any()  # the switch is inside the scan
    assert np.abs(np.diff(vals)).max() < 20 * (ts[1] - ts[0])


def test_tau_to_zero_recovers_the_hard_solution_and_record():
    raw, src, prj, h = setup()
    Th, _, st, _ = O.solve_gs(prj, src, h, 1e-6)
    assert st == O.OK
    T0, _, st0 = O.solve_softmin(prj, src, h, 1e-6, 0.0)
    assert st0 == O.OK and np.array_equal(T0, Th)
    Ts, _, sts = O.solve_softmin(prj, src, h, 1e-6, 1e-10 * h)
    assert sts == O.OK
    assert np.abs(Ts - Th).max() <= 1e-8 * Th.max()
    # record: weights and partials of the hard update away from near-ties
    rec = O.record(prj, src, h, 1e-6, Th)
    wnb, dth = O.softmin_record(prj, src, h, 1e-6, Th, 1e-10 * h)
    tie = rec["margin"] < 1e-6 * Th.max()
    keep = (rec["id"] != 0) & ~tie
    k = (rec["id"] & 7).astype(int)
    first = wnb[k, np.arange(k.shape[0])[:, None], np.arange(k.shape[1])[None, :]]
    # (a degenerate two-point stencil, barycentric weight ~1e-6, sits within
    # tau of the one-point it equals and keeps a share of the weight)
    assert np.allclose(first[keep], rec["w1"][keep], atol=1e-5)
    assert np.allclose(dth[:, keep], rec["dT"][:, keep], rtol=1e-5, atol=1e-9)
    assert np.allclose(wnb.sum(axis=0)[keep], 1.0, atol=1e-12)


def test_relaxed_solution_is_below_and_decreases_with_tau():
    raw, src, prj, h = setup()
    Th, _, _, _ = O.solve_gs(prj, src, h, 1e-6)
    prev = Th
    for rel in (0.005, 0.02, 0.05):
        tau = rel * h
        Ts, _, st = O.solve_softmin(prj, src, h, 1e-6, tau)
        assert st == O.OK
        fin = np.isfinite(Th)
        assert np.array_equal(np.isfinite(Ts), fin)
        assert np.all(Ts[fin] <= prev[fin] + 1e-13)
        prev = Ts
        # each node: within tau log 16 below its candidate minimum at Ts
        res = O.residual(prj, src, h, 1e-6, Ts)  # T - min candidate
        assert np.all(res[fin] <= 1e-12) and np.all(res[fin] >= -tau * np.log(16.0) - 1e-12)


def test_weights_sum_to_one_and_adjoint_conserves_mass():
    raw, src, prj, h = setup()
    tau = 0.05 * h
    Ts, _, st = O.solve_softmin(prj, src, h, 1e-6, tau)
    assert st == O.OK
    wnb, dth = O.softmin_record(prj, src, h, 1e-6, Ts, tau)
    reached = np.isfinite(Ts) & (src == 0)
    assert np.allclose(wnb.sum(axis=0)[reached], 1.0, atol=1e-12)
    assert np.all(wnb >= -1e-15)
    g = R.sparse_loss_grad(*src.shape, 0.2, seed=1).astype(np.float64)
    lam, grad, passes = O.softmin_adjoint(src, Ts, wnb, dth, g)
    assert lam[src == 1].sum() == pytest.approx(g[np.isfinite(Ts)].sum(), rel=1e-10)


def _loss(raw, src, h, tau, g, eps=1e-6, delta=0.05):
    prj, _ = O.project(raw, eps, delta)
    T, _, st = O.solve_softmin(prj, src, h, eps, tau, tol=1e-15, max_iter=5000)
    assert st == O.OK
    return float(np.sum(np.where(np.isfinite(T), g * T, 0.0)))


def test_adjoint_matches_finite_differences():
    raw, src, prj, h = setup(n=16)
    tau = 0.05 * h
    g = R.sparse_loss_grad(16, 16, 0.3, seed=2).astype(np.float64)
    out = O.softmin_solve_and_grad(raw, src, h, 1e-6, 0.05, g, tau)
    rng = np.random.default_rng(4)
    errs = []
    for _ in range(24):
        c, i, j = int(rng.integers(0, 5)), int(rng.integers(0, 16)), int(rng.integers(0, 16))
        if src[i, j]:
            continue
        # step 1e-4: the FP64 solve stops at 1e-15, so a smaller step's
        # quotient is mostly rounding noise for entries of ~1e-6
        step = 1e-4 * max(1.0, abs(raw[c, i, j]))
        rp, rm = raw.copy(), raw.copy()
        rp[c, i, j] += step
        rm[c, i, j] -= step
        fd = (_loss(rp, src, h, tau, g) - _loss(rm, src, h, tau, g)) / (2 * step)
        an = out["graw"][c, i, j]
        # relative to the entry, with a floor of 1e-6 of the largest entry
        # (below it the quotient is rounding noise of the FP64 loss)
        errs.append(abs(fd - an) / max(1e-6 * np.abs(out["graw"]).max(), abs(an), abs(fd)))
    assert max(errs) < 1e-4, errs


def test_gradient_is_smooth_across_a_stencil_switch():
    """Two sources at the ends of the middle row of an isotropic 9 x 9 grid:
    the middle node is reached equally from both sides, so the hard solution
    switches its stencil there and T(middle) has a kink in the metric of a
    node on one side.  The soft solution's derivative, from its adjoint,
    matches a central difference whose step crosses the switch."""
    n = 9
    h = 1.0 / (n - 1)
    raw = np.zeros((5, n, n))
    raw[0] = raw[2] = 1.0
    src = np.zeros((n, n), np.uint8)
    src[4, 0] = src[4, n - 1] = 1
    g = np.zeros((n, n))
    g[4, 4] = 1.0
    c, i, j = 0, 4, 2  # L11 of a node on the left path
    tau = 0.05 * h
    out = O.softmin_solve_and_grad(raw, src, h, 0.0, 0.05, g, tau)
    step = 1e-5
    rp, rm = raw.copy(), raw.copy()
    rp[c, i, j] += step
    rm[c, i, j] -= step
    fd = (_loss(rp, src, h, tau, g, eps=0.0) - _loss(rm, src, h, tau, g, eps=0.0)) / (2 * step)
    assert out["graw"][c, i, j] == pytest.approx(fd, rel=1e-5)
    # the hard solution has a kink there: one-sided slopes differ
    def hard(r):
        prj, _ = O.project(r, 0.0, 0.05)
        T, _, _, _ = O.solve_gs(prj, src, h, 0.0)
        return T[4, 4]
    up = (hard(rp) - hard(raw)) / step
    down = (hard(raw) - hard(rm)) / step
    assert abs(up - down) > 0.1 * max(abs(up), abs(down))


def test_too_large_tau_has_no_finite_fixed_point():
    """With tau log(16) above the edge costs the relaxed values run to -inf:
    the solve reports non-convergence instead of a result."""
    raw, src, prj, h = setup()
    Ts, _, st = O.solve_softmin(prj, src, h, 1e-6, 2.0 * h, max_iter=300)
    assert st == O.ERR_NOT_CONVERGED
