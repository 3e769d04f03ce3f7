"""RFSolve (torch.autograd.Function over the CUDA path) against the FP64
oracle's implicit gradients, and the inverse-problem driver.

The oracle's gradients are themselves pinned to finite differences
(tests/test_oracle_adjoint.py), so agreement here checks the CUDA autograd
path against FD and the FP64 adjoint at once.
"""
import numpy as np
import pytest

import oracle as O
import rf_inputs as R
from gpu_util import GRAD_TOL, flip_mask, rel_l2, require_gpu, to_dev, torch
from paper_2603_00035_gb300 import api
from paper_2603_00035_gb300.autograd import rf_solve
from paper_2603_00035_gb300.inverse import run_inverse

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def crop_case(n_full=2048, n=256, seed=0):
    """Top-left n x n crop of the 2048^2 inverse-problem fields, re-solved
    standalone with 3 seeded sources inside the crop."""
    c = R.config_inverse(n=n_full, seed=seed)
    raw = np.ascontiguousarray(c["raw"][:, :n, :n])
    src = R.random_sources(n, n, 3, seed=seed + 11, margin=4)
    obs = R.observation_mask(n, n, 0.05, seed=seed)
    return raw, src, obs, c["h"], c["eps"], c["delta"]


def target_times(raw_shape, src, h, eps, delta, seed):
    """T-hat from a second field solved by the oracle (FP64)."""
    ny, nx = src.shape
    raw2 = R.randers_fields(ny, nx, h, 16, seed + 1000, omega="unit", omega_scale=0.3)
    pr, _ = O.project(raw2, eps, delta)
    T2, _, st, _ = O.solve_gs(pr, src, h, eps)
    assert st == O.OK
    return T2


@pytest.mark.parametrize("which", ["config1", "crop256"])
@pytest.mark.parametrize("algo", ["tiles", "ordered", "sweep"])
def test_rfsolve_gradients_match_oracle(which, algo):
    if which == "config1":
        c = R.config1()
        raw, src, h, eps, delta = c["raw"], c["src"], c["h"], c["eps"], c["delta"]
        obs = R.observation_mask(64, 64, 0.05, seed=0)
    else:
        raw, src, obs, h, eps, delta = crop_case()
    That = target_times(raw.shape, src, h, eps, delta, seed=3)
    # GPU: autograd through RFSolve
    raw_t = to_dev(raw, torch.float32).requires_grad_(True)
    src_t = to_dev(src, torch.uint8)
    obs_t = to_dev(obs, torch.float32)
    That_t = to_dev(That, torch.float32)
    T = rf_solve(raw_t, src_t, h, eps, delta, algo)
    loss = 0.5 * (obs_t * (T - That_t) ** 2).sum()
    loss.backward()
    assert api.Context.get(0).stats()["status"] == 0
    g_gpu = raw_t.grad.detach().cpu().numpy()
    # oracle: same loss, FP64 throughout
    proj, _ = O.project(raw, eps, delta)
    To, _, _, _ = O.solve_gs(proj, src, h, eps)
    g_o = obs * (To - That)
    orc = O.solve_and_grad(raw.astype(np.float64), src, h, eps, delta, g_o)
    rec_g = api.rf_sweep_forward(api.rf_project(to_dev(raw, torch.float32), eps, delta)[0], eps, src_t, h)[1]
    gpu_like = dict(rec_np=dict(id=rec_g.id.cpu().numpy(), w1=rec_g.w1.cpu().numpy()))
    flips, _ = flip_mask(gpu_like, orc)
    err = rel_l2(g_gpu, orc["graw"], ~flips)
    assert err < GRAD_TOL, (which, algo, err, int(flips.sum()))
    # loss values agree too
    assert float(loss.detach()) == pytest.approx(0.5 * float((obs * (To - That) ** 2).sum()), rel=1e-4)


def test_inverse_problem_reduces_loss_and_error():
    n = 256
    c = R.config_inverse(n=n, seed=5)
    raw_true = to_dev(c["raw"], torch.float32)
    src = to_dev(c["src"], torch.uint8)
    obs = to_dev(R.observation_mask(n, n, 0.05, seed=5), torch.uint8)
    out = run_inverse(raw_true, src, obs, c["h"], steps=40, log_every=1)
    losses = [l for _, l in out["loss_history"]]
    assert losses[-1] < 0.3 * losses[0], losses[::8]
    assert out["final_loss"] < losses[0]
    assert np.isfinite(out["rel_err_metric"]) and np.isfinite(out["rel_err_drift"])
