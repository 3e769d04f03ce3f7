"""The streamed forward sweep evaluates the two-point update (Eq. 2,
App. A) in a rearranged closed form; this checks the rearrangement against
the oracle's update in the paper's notation (FP64, CPU).

With S_n = T_n - w.m_n, d = S_b - S_a, e_xy = m_x^T M m_y and
aa = |m_a - m_b|^2_M:

    T0 = S_a + C d + sqrt(P - Q d^2),  C = (e_aa - e_ab) / aa,
    P = det E / aa,  Q = det E / aa^2,

valid iff (e_ab - e_bb) / |m_b| < d < (e_aa - e_ab) / |m_a| (the segment
minimiser is interior, i.e. both barycentric weights >= 0) and both donors
are earlier than T0.
"""
import numpy as np

import oracle as O

DX = [-1, -1, -1, 0, 1, 1, 1, 0]
DY = [1, 0, -1, -1, -1, 0, 1, 1]


def cone_candidate(Tn, h, M, w, k):
    a, b = k, (k + 1) % 8
    m = [np.array([DX[n], DY[n]], float) * h for n in range(8)]
    S = [Tn[n] - w @ m[n] for n in range(8)]
    eaa, ebb, eab = m[a] @ M @ m[a], m[b] @ M @ m[b], m[a] @ M @ m[b]
    aa = (m[a] - m[b]) @ M @ (m[a] - m[b])
    dete = np.linalg.det(M) * h ** 4
    lo, hi = (eab - ebb) / np.sqrt(ebb), (eaa - eab) / np.sqrt(eaa)
    with np.errstate(invalid="ignore"):
        d = S[b] - S[a]
        q = dete / aa - dete / aa ** 2 * d * d
        T0 = S[a] + (eaa - eab) / aa * d + np.sqrt(q) if q >= 0 else np.nan
        ok = bool(lo < d < hi) and max(Tn[a], Tn[b]) < T0
    return ok, T0, min(abs(d - lo), abs(d - hi)) if np.isfinite(d) else np.inf


def test_cone_form_matches_oracle_update():
    rng = np.random.default_rng(0)
    checked = valid = 0
    for _ in range(3000):
        th = rng.uniform(0, np.pi)
        ra, rb = rng.uniform(0.5, 2.0, 2)
        c, s = np.cos(th), np.sin(th)
        M = np.array([[ra * ra * c * c + rb * rb * s * s, (ra * ra - rb * rb) * c * s],
                      [(ra * ra - rb * rb) * c * s, ra * ra * s * s + rb * rb * c * c]])
        w = rng.normal(size=2)
        w *= rng.uniform(0, 0.9) / np.sqrt(w @ np.linalg.solve(M, w))
        h = 0.01
        Tn = rng.uniform(0, 0.05, 8)
        Tn[rng.random(8) < 0.2] = np.inf
        r = O.cell_eval(Tn, h, M[0, 0], M[0, 1], M[1, 1], w[0], w[1])
        for k in range(8):
            ok, T0, margin = cone_candidate(Tn, h, M, w, k)
            if margin < 1e-9:
                continue  # on the cone boundary the two forms may round differently
            checked += 1
            assert ok == bool(r["two_ok"][k]), (k, ok, r["two_ok"][k])
            if ok:
                valid += 1
                assert abs(T0 - r["two"][k]) <= 1e-12 * max(1.0, abs(T0))
    assert checked > 20000 and valid > 1000
