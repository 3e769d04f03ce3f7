"""RF_ADJ_LEVELS (DAG-depth pass, then a level-synchronous gather) on the GPU.

The level schedule changes the order in which multipliers are finished, not
the sum each node forms (children in the fixed neighbour order), so lambda
and the gradients must equal RF_ADJ_ORDERED's bit for bit; the level count
reported in the stats must be the depth of the record's donor DAG, counted
here on the host; and against the FP64 oracle the usual gradient tolerance
holds (App. A, Alg. 2).
"""
import numpy as np
import pytest

import rf_inputs as R
from gpu_util import GRAD_TOL, api, flip_mask, gpu_path, oracle_path, rel_l2, require_gpu, to_dev, torch

pytestmark = pytest.mark.gpu

# Fig. 4(a): neighbours counter-clockwise from the upper-left, (dx, dy) with +y = +i
RING = [(-1, 1), (-1, 0), (-1, -1), (0, -1), (1, -1), (1, 0), (1, 1), (0, 1)]


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def ragged_case():
    ny, nx = 203, 141
    h = 1.0 / 202
    return dict(raw=R.randers_fields(ny, nx, h, 8, seed=9, omega="field", omega_max=1.0),
                src=R.random_sources(ny, nx, 3, seed=9), h=h, eps=1e-6, delta=0.3,
                g=R.sparse_loss_grad(ny, nx, 0.05, seed=9))


CASES = {"config1": R.config1, "ragged": ragged_case, "config2": R.config2}


def dag_depth(T, ids):
    """Number of levels of the donor DAG: a node without donors has level 0,
    any other 1 + the largest level of its donors (one-point record 0x10|k:
    neighbour k; two-point 0x20|k: neighbours k and k+1).  0 if no node is
    reached."""
    ny, nx = T.shape
    Tf, idf = T.ravel(), ids.ravel()
    reached = np.flatnonzero(np.isfinite(Tf))
    level = np.full(Tf.size, -1, np.int64)
    for p in reached[np.argsort(Tf[reached], kind="stable")]:
        i, j = divmod(int(p), nx)
        d = int(idf[p])
        donors = [d & 7] if d & 0x10 else ([d & 7, ((d & 7) + 1) % 8] if d & 0x20 else [])
        lv = 0
        for k in donors:
            dx, dy = RING[k]
            q = (i + dy) * nx + (j + dx)
            assert level[q] >= 0, "donor not finished before its child"
            lv = max(lv, int(level[q]) + 1)
        level[p] = lv
    return int(level.max()) + 1 if reached.size else 0


@pytest.mark.parametrize("name", list(CASES))
def test_levels_equal_ordered_bitwise(name):
    c = CASES[name]()
    gpu = gpu_path(c["raw"], c["src"], c["h"], c["eps"], c["delta"], c["g"], algo="ordered")
    src = to_dev(c["src"], torch.uint8)
    T = to_dev(gpu["T"], torch.float32)
    g = to_dev(c["g"], torch.float32)
    ctx = api.Context.get(0)
    gproj, lam = api.rf_adjoint(src, T, gpu["rec"], g, algo="levels")
    st = ctx.stats()
    assert st["status"] == 0, st
    assert np.array_equal(lam.cpu().numpy().view(np.uint32), gpu["lam"].view(np.uint32))
    assert np.array_equal(gproj.cpu().numpy().view(np.uint32), gpu["gproj"].view(np.uint32))
    if name != "config2":  # the host count walks every node in Python
        assert st["adj_sweeps"] == dag_depth(gpu["T"], gpu["rec_np"]["id"])
    orc = oracle_path(c["raw"], c["src"], c["h"], c["eps"], c["delta"], c["g"])
    flips, _ = flip_mask(gpu, orc)
    assert rel_l2(gproj.cpu().numpy(), orc["gproj"], ~flips) < GRAD_TOL


def test_levels_on_oracle_record():
    """The level gather fed the oracle's record: lambda and the gradients
    match the FP64 back-substitution to float32 accuracy."""
    c = R.config1()
    orc = oracle_path(c["raw"], c["src"], c["h"], c["eps"], c["delta"], c["g"])
    rec = api.Record(to_dev(orc["rec"]["id"], torch.uint8), to_dev(orc["rec"]["w1"], torch.float32),
                     to_dev(orc["rec"]["dT"], torch.float32))
    T = to_dev(orc["T"], torch.float32)
    src = to_dev(c["src"], torch.uint8)
    g = to_dev(np.where(np.isfinite(orc["T"]), c["g"], 0.0), torch.float32)
    gproj, lam = api.rf_adjoint(src, T, rec, g, algo="levels")
    st = api.Context.get(0).stats()
    assert st["status"] == 0
    assert st["adj_sweeps"] == dag_depth(orc["T"], orc["rec"]["id"])
    assert rel_l2(lam.cpu().numpy(), orc["lam"]) < 1e-5
    assert rel_l2(gproj.cpu().numpy(), orc["gproj"]) < 1e-5


def test_levels_full_size_equal_ordered():
    """The 2048^2 inverse-problem workload: the level schedule reproduces
    the ordered gather bit for bit."""
    c = R.config_inverse(2048)
    ctx = api.Context.get(0)
    raw = to_dev(c["raw"], torch.float32)
    src = to_dev(c["src"], torch.uint8)
    g = to_dev(c["g"], torch.float32)
    proj, _ = api.rf_project(raw, c["eps"], c["delta"])
    T, rec = api.rf_sweep_forward(proj, c["eps"], src, c["h"])
    assert ctx.stats()["status"] == 0
    g1, l1 = api.rf_adjoint(src, T, rec, g, algo="ordered")
    assert ctx.stats()["status"] == 0
    g2, l2 = api.rf_adjoint(src, T, rec, g, algo="levels")
    st = ctx.stats()
    assert st["status"] == 0 and st["adj_sweeps"] > 100
    assert torch.equal(l1.view(torch.int32), l2.view(torch.int32))
    assert torch.equal(g1.view(torch.int32), g2.view(torch.int32))


def test_levels_single_node_and_no_source():
    ctx = api.Context.get(0)
    # 1 x 1 source: one level, zero gradient, lambda = g
    T = torch.zeros((1, 1), device="cuda")
    rec = api.Record(torch.zeros((1, 1), dtype=torch.uint8, device="cuda"), torch.zeros((1, 1), device="cuda"),
                     torch.zeros((5, 1, 1), device="cuda"))
    g = torch.full((1, 1), 0.5, device="cuda")
    gproj, lam = api.rf_adjoint(torch.ones((1, 1), dtype=torch.uint8, device="cuda"), T, rec, g, algo="levels")
    st = ctx.stats()
    assert st["status"] == 0 and st["adj_sweeps"] == 1
    assert lam.item() == 0.5 and (gproj == 0).all()
    # nothing reached: no level, everything zero
    ny, nx = 20, 30
    T = torch.full((ny, nx), float("inf"), device="cuda")
    rec = api.Record(torch.zeros((ny, nx), dtype=torch.uint8, device="cuda"), torch.zeros((ny, nx), device="cuda"),
                     torch.zeros((5, ny, nx), device="cuda"))
    g = torch.ones((ny, nx), device="cuda")
    gproj, lam = api.rf_adjoint(torch.zeros((ny, nx), dtype=torch.uint8, device="cuda"), T, rec, g, algo="levels")
    st = ctx.stats()
    assert st["status"] == 0 and st["adj_sweeps"] == 0
    assert (lam == 0).all() and (gproj == 0).all()


def test_levels_timeout_returns_cleanly():
    """A zero wait bound makes the depth pass (or the first level barrier)
    give up: RF_ERR_TIMEOUT, and the next call with a normal bound works."""
    c = R.config2()
    ctx = api.Context(0)
    raw = to_dev(c["raw"], torch.float32)
    src = to_dev(c["src"], torch.uint8)
    proj, _ = api.rf_project(raw, c["eps"], c["delta"], ctx=ctx)
    T, rec = api.rf_sweep_forward(proj, c["eps"], src, c["h"], ctx=ctx)
    assert ctx.stats()["status"] == 0
    g = to_dev(c["g"], torch.float32)
    ctx.set_timeout(0)
    api.rf_adjoint(src, T, rec, g, algo="levels", ctx=ctx)
    assert ctx.stats()["status"] == 4  # RF_ERR_TIMEOUT
    ctx.set_timeout(2_000_000_000)
    g1, _ = api.rf_adjoint(src, T, rec, g, algo="levels", ctx=ctx)
    assert ctx.stats()["status"] == 0
    g2, _ = api.rf_adjoint(src, T, rec, g, algo="ordered", ctx=ctx)
    assert torch.equal(g1.view(torch.int32), g2.view(torch.int32))
