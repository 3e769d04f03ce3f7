"""Soft-min relaxation on the GPU (rf_softmin_forward / _record / _adjoint,
through the C ABI) against the FP64 oracle's soft-min solve, record and
adjoint on the same seeded inputs (Sec. 3.3 names the relaxation; the
formula -- T = -tau log sum_k exp(-c_k/tau) over the 8 stencil segment
minima -- is the build's reading, pinned in test_oracle_softmin.py)."""
import numpy as np
import pytest

import oracle as O
import rf_inputs as R
from gpu_util import FWD_TOL, GRAD_TOL, api, rel_l2, require_gpu, to_dev, torch
from paper_2603_00035_gb300 import _lib as L
from paper_2603_00035_gb300.autograd import SoftSolve

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def ragged():
    ny, nx = 75, 53
    h = 1.0 / 74
    return dict(raw=R.randers_fields(ny, nx, h, 8, seed=12, omega="unit", omega_scale=0.3),
                src=R.random_sources(ny, nx, 3, seed=12), h=h, eps=1e-6, delta=0.05,
                g=R.sparse_loss_grad(ny, nx, 0.1, seed=12))


CASES = {"config1": R.config1, "ragged": ragged}


@pytest.mark.parametrize("variant", ["tiles", "tiled1"])  # tile queue; Jacobi over the grid
@pytest.mark.parametrize("which", list(CASES))
@pytest.mark.parametrize("rel_tau", [0.002, 0.05])
def test_softmin_solve_record_and_gradient_match_oracle(which, rel_tau, variant):
    c = CASES[which]()
    tau = rel_tau * c["h"]
    orc = O.softmin_solve_and_grad(c["raw"].astype(np.float64), c["src"], c["h"], c["eps"], c["delta"],
                                   c["g"].astype(np.float64), tau)
    assert orc["status"] == O.OK
    raw = to_dev(c["raw"], torch.float32)
    src = to_dev(c["src"], torch.uint8)
    proj, clip = api.rf_project(raw, c["eps"], c["delta"])
    T = api.rf_softmin_forward(proj, c["eps"], src, c["h"], tau, opts=api.make_opts(variant=variant))
    st = api.Context.get(0).stats()
    assert st["status"] == 0 and st["converged"], st
    Tg, To = T.cpu().numpy(), orc["T"]
    assert np.array_equal(np.isfinite(Tg), np.isfinite(To))
    fin = np.isfinite(To)
    assert np.abs(Tg[fin] - To[fin]).max() <= FWD_TOL * To[fin].max()
    wnb, dT = api.rf_softmin_record(proj, c["eps"], src, c["h"], T, tau)
    assert rel_l2(wnb.cpu().numpy(), orc["wnb"]) < 1e-3
    assert rel_l2(dT.cpu().numpy(), orc["dth"]) < 1e-3
    reached = fin & (c["src"] == 0)
    assert np.allclose(wnb.cpu().numpy().sum(axis=0)[reached], 1.0, atol=1e-5)
    g = to_dev(np.where(fin, c["g"], 0.0).astype(np.float32), torch.float32)
    gproj, lam = api.rf_softmin_adjoint(src, T, wnb, dT, g)
    assert api.Context.get(0).stats()["status"] == 0
    assert rel_l2(lam.cpu().numpy(), orc["lam"]) < GRAD_TOL
    assert rel_l2(gproj.cpu().numpy(), orc["gproj"]) < GRAD_TOL
    # mass conservation: the sources collect every observation's weight
    assert lam.cpu().numpy()[c["src"] == 1].sum() == pytest.approx(float(g.sum()), rel=1e-4)
    graw = api.rf_project_backward(raw, clip, c["eps"], c["delta"], gproj)
    assert rel_l2(graw.cpu().numpy(), orc["graw"]) < GRAD_TOL


def test_softmin_with_tau_zero_is_the_hard_solve():
    c = R.config2()
    raw = to_dev(c["raw"], torch.float32)
    src = to_dev(c["src"], torch.uint8)
    proj, _ = api.rf_project(raw, c["eps"], c["delta"])
    Ts = api.rf_softmin_forward(proj, c["eps"], src, c["h"], 0.0)
    assert api.Context.get(0).stats()["status"] == 0
    Th, _ = api.rf_sweep_forward(proj, c["eps"], src, c["h"], record=False)
    assert api.Context.get(0).stats()["status"] == 0
    assert (Ts - Th).abs().max().item() <= FWD_TOL * Th.max().item()


def test_softmin_autograd_across_a_stencil_switch():
    """The isotropic 9 x 9 grid with a source at each end of the middle row:
    the middle node switches stencils there; SoftSolve's gradient with
    respect to a metric entry on one side matches the oracle's soft adjoint
    (which itself matches central differences across the switch)."""
    n = 9
    h = 1.0 / (n - 1)
    raw = np.zeros((5, n, n), np.float32)
    raw[0] = raw[2] = 1.0
    src = np.zeros((n, n), np.uint8)
    src[4, 0] = src[4, n - 1] = 1
    g = np.zeros((n, n), np.float32)
    g[4, 4] = 1.0
    tau = 0.05 * h
    orc = O.softmin_solve_and_grad(raw.astype(np.float64), src, h, 0.0, 0.05, g.astype(np.float64), tau)
    x = to_dev(raw, torch.float32).requires_grad_(True)
    T = SoftSolve.apply(x, to_dev(src, torch.uint8), h, tau, 0.0, 0.05, None)
    (T * to_dev(g, torch.float32)).sum().backward()
    gg = x.grad.cpu().numpy()
    assert gg[0, 4, 2] == pytest.approx(orc["graw"][0, 4, 2], rel=1e-3)
    assert rel_l2(gg, orc["graw"]) < GRAD_TOL


def test_too_large_tau_is_reported_not_run_forever():
    """tau log 8 above the edge costs: no finite fixed point; the solve stops
    as soon as a node goes negative and reports RF_ERR_NOT_CONVERGED."""
    c = R.config1()
    raw = to_dev(c["raw"], torch.float32)
    src = to_dev(c["src"], torch.uint8)
    proj, _ = api.rf_project(raw, c["eps"], c["delta"])
    for variant in ("tiles", "tiled1"):
        api.rf_softmin_forward(proj, c["eps"], src, c["h"], 2.0 * c["h"], opts=api.make_opts(variant=variant))
        st = api.Context.get(0).stats()
        assert st["status"] == L.RF_ERR_NOT_CONVERGED, variant
        assert st["sweeps"] < 64 * 64, variant  # stopped early, not at the iteration cap


def test_softmin_tile_queue_equals_jacobi_at_512():
    """The 512^2 workload: the tile queue and the Jacobi iterations solve the
    same relaxed system (within the stopping tolerance), deterministically."""
    c = R.config2()
    tau = 0.05 * c["h"]
    raw = to_dev(c["raw"], torch.float32)
    src = to_dev(c["src"], torch.uint8)
    proj, _ = api.rf_project(raw, c["eps"], c["delta"])
    Tt = api.rf_softmin_forward(proj, c["eps"], src, c["h"], tau, opts=api.make_opts(variant="tiles"))
    st = api.Context.get(0).stats()
    assert st["status"] == 0 and st["converged"], st
    Tt2 = api.rf_softmin_forward(proj, c["eps"], src, c["h"], tau, opts=api.make_opts(variant="tiles"))
    assert torch.equal(Tt, Tt2)
    Tj = api.rf_softmin_forward(proj, c["eps"], src, c["h"], tau, opts=api.make_opts(variant="tiled1"))
    assert api.Context.get(0).stats()["status"] == 0
    assert (Tt - Tj).abs().max().item() <= FWD_TOL * Tj.max().item()
