"""RF_ADJ_TILES (16 x 16 tiles by decreasing latest T, the dependency chain
inside a tile followed in shared memory) on the GPU.

The tile schedule changes only when each multiplier is formed, not the sum
(children in the fixed neighbour order, the same fused multiply-adds), so
lambda and the gradients must equal RF_ADJ_ORDERED's bit for bit -- also
when every waiting tile yields its CTA at once (park 0), which sends tiles
through the retry ring -- and against the FP64 oracle the usual gradient
tolerance holds (App. A, Alg. 2).
"""
import numpy as np
import pytest

import rf_inputs as R
from gpu_util import GRAD_TOL, api, flip_mask, gpu_path, oracle_path, rel_l2, require_gpu, to_dev, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def ragged_case():
    ny, nx = 203, 141
    h = 1.0 / 202
    return dict(raw=R.randers_fields(ny, nx, h, 8, seed=9, omega="field", omega_max=1.0),
                src=R.random_sources(ny, nx, 3, seed=9), h=h, eps=1e-6, delta=0.3,
                g=R.sparse_loss_grad(ny, nx, 0.05, seed=9))


def strip_case():
    # one tile high, many tiles wide, a ragged last tile; sources at both ends
    ny, nx = 13, 301
    h = 1.0 / 300
    src = np.zeros((ny, nx), np.uint8)
    src[0, 0] = src[ny - 1, nx - 1] = 1
    return dict(raw=R.randers_fields(ny, nx, h, 4, seed=5, omega="field", omega_max=0.8), src=src, h=h, eps=1e-6,
                delta=0.3, g=R.sparse_loss_grad(ny, nx, 0.2, seed=5))


CASES = {"config1": R.config1, "ragged": ragged_case, "strip": strip_case, "config2": R.config2}


def bits(t):
    return t.cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("park_ns", [100_000, 0])
@pytest.mark.parametrize("name", list(CASES))
def test_tiles_equal_ordered_bitwise(name, park_ns):
    c = CASES[name]()
    gpu = gpu_path(c["raw"], c["src"], c["h"], c["eps"], c["delta"], c["g"], algo="ordered")
    src = to_dev(c["src"], torch.uint8)
    T = to_dev(gpu["T"], torch.float32)
    g = to_dev(c["g"], torch.float32)
    ctx = api.Context(0)
    ctx.set_adjoint_park(park_ns)
    gproj, lam = api.rf_adjoint(src, T, gpu["rec"], g, algo="tiles", ctx=ctx)
    st = ctx.stats()
    assert st["status"] == 0, st
    assert np.array_equal(bits(lam), gpu["lam"].view(np.uint32))
    assert np.array_equal(bits(gproj), gpu["gproj"].view(np.uint32))
    if park_ns == 0 and name in ("ragged", "config2"):
        assert st["adj_sweeps"] > 0  # tiles did yield and were retried
    if park_ns == 0:
        orc = oracle_path(c["raw"], c["src"], c["h"], c["eps"], c["delta"], c["g"])
        flips, _ = flip_mask(gpu, orc)
        assert rel_l2(gproj.cpu().numpy(), orc["gproj"], ~flips) < GRAD_TOL


def test_tiles_on_oracle_record():
    """The tile gather fed the oracle's record: lambda and the gradients
    match the FP64 back-substitution to float32 accuracy."""
    c = R.config1()
    orc = oracle_path(c["raw"], c["src"], c["h"], c["eps"], c["delta"], c["g"])
    rec = api.Record(to_dev(orc["rec"]["id"], torch.uint8), to_dev(orc["rec"]["w1"], torch.float32),
                     to_dev(orc["rec"]["dT"], torch.float32))
    T = to_dev(orc["T"], torch.float32)
    src = to_dev(c["src"], torch.uint8)
    g = to_dev(np.where(np.isfinite(orc["T"]), c["g"], 0.0), torch.float32)
    gproj, lam = api.rf_adjoint(src, T, rec, g, algo="tiles")
    assert api.Context.get(0).stats()["status"] == 0
    assert rel_l2(lam.cpu().numpy(), orc["lam"]) < 1e-5
    assert rel_l2(gproj.cpu().numpy(), orc["gproj"]) < 1e-5


def test_tiles_full_size_equal_ordered():
    """The 2048^2 inverse-problem workload: the tile schedule reproduces the
    ordered gather bit for bit, repeatedly (epoch tags across calls)."""
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
    for _ in range(3):
        g2, l2 = api.rf_adjoint(src, T, rec, g, algo="tiles")
        assert ctx.stats()["status"] == 0
        assert torch.equal(l1.view(torch.int32), l2.view(torch.int32))
        assert torch.equal(g1.view(torch.int32), g2.view(torch.int32))


def test_tiles_single_node_and_no_source():
    ctx = api.Context.get(0)
    T = torch.zeros((1, 1), device="cuda")
    rec = api.Record(torch.zeros((1, 1), dtype=torch.uint8, device="cuda"), torch.zeros((1, 1), device="cuda"),
                     torch.zeros((5, 1, 1), device="cuda"))
    g = torch.full((1, 1), 0.5, device="cuda")
    gproj, lam = api.rf_adjoint(torch.ones((1, 1), dtype=torch.uint8, device="cuda"), T, rec, g, algo="tiles")
    assert ctx.stats()["status"] == 0
    assert lam.item() == 0.5 and (gproj == 0).all()
    ny, nx = 20, 30
    T = torch.full((ny, nx), float("inf"), device="cuda")
    rec = api.Record(torch.zeros((ny, nx), dtype=torch.uint8, device="cuda"), torch.zeros((ny, nx), device="cuda"),
                     torch.zeros((5, ny, nx), device="cuda"))
    g = torch.ones((ny, nx), device="cuda")
    gproj = torch.full((5, ny, nx), 7.0, device="cuda")
    gproj, lam = api.rf_adjoint(torch.zeros((ny, nx), dtype=torch.uint8, device="cuda"), T, rec, g, algo="tiles",
                                dLdproj5=gproj)
    assert ctx.stats()["status"] == 0
    assert (lam == 0).all() and (gproj == 0).all()


def test_tiles_timeout_returns_cleanly():
    """A zero wait bound makes the first stalled tile give up:
    RF_ERR_TIMEOUT, and the next call with a normal bound works."""
    c = R.config2()
    ctx = api.Context(0)
    raw = to_dev(c["raw"], torch.float32)
    src = to_dev(c["src"], torch.uint8)
    proj, _ = api.rf_project(raw, c["eps"], c["delta"], ctx=ctx)
    T, rec = api.rf_sweep_forward(proj, c["eps"], src, c["h"], ctx=ctx)
    assert ctx.stats()["status"] == 0
    g = to_dev(c["g"], torch.float32)
    ctx.set_timeout(0)
    api.rf_adjoint(src, T, rec, g, algo="tiles", ctx=ctx)
    assert ctx.stats()["status"] == 4  # RF_ERR_TIMEOUT
    ctx.set_timeout(2_000_000_000)
    g1, _ = api.rf_adjoint(src, T, rec, g, algo="tiles", ctx=ctx)
    assert ctx.stats()["status"] == 0
    g2, _ = api.rf_adjoint(src, T, rec, g, algo="ordered", ctx=ctx)
    assert torch.equal(g1.view(torch.int32), g2.view(torch.int32))


@pytest.mark.parametrize("algo", ["tiles", "ordered"])
def test_adjoint_graph_replay_with_new_inputs(algo):
    """rf_adjoint captured in a CUDA graph: every replay tags its state words
    anew (a device-side epoch), so a replay after dL/dT changed gives what a
    direct call with the new dL/dT gives, bit for bit (a tag fixed at
    capture would let the replay reuse the previous multipliers)."""
    c = R.config2()
    ctx = api.Context(0)
    raw = to_dev(c["raw"], torch.float32)
    src = to_dev(c["src"], torch.uint8)
    proj, _ = api.rf_project(raw, c["eps"], c["delta"], ctx=ctx)
    T, rec = api.rf_sweep_forward(proj, c["eps"], src, c["h"], ctx=ctx)
    g = to_dev(c["g"], torch.float32)
    ny, nx = T.shape
    gproj = torch.empty((5, ny, nx), device="cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        api.rf_adjoint(src, T, rec, g, algo=algo, dLdproj5=gproj, ctx=ctx, stream=s)  # sizes the workspace
        s.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=s):
            _, lam_g = api.rf_adjoint(src, T, rec, g, algo=algo, dLdproj5=gproj, ctx=ctx, stream=s)
    torch.cuda.current_stream().wait_stream(s)
    for k in range(3):
        if k:
            g.copy_(to_dev(R.sparse_loss_grad(ny, nx, 0.05, seed=100 + k), torch.float32))
        want_g, want_l = api.rf_adjoint(src, T, rec, g, algo=algo, ctx=ctx)
        torch.cuda.synchronize()
        graph.replay()
        torch.cuda.synchronize()
        assert torch.equal(gproj, want_g) and torch.equal(lam_g, want_l), k
        assert ctx.stats()["status"] == 0
