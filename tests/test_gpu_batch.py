"""rf_batch_solve: many grids of uneven size (square and 2:1) and source
count in one persistent launch, checked against the single-grid CUDA path
(same discrete system, same sweep schedule) and the FP64 oracle, and
replayed from a CUDA graph."""
import numpy as np
import pytest

import oracle as O
import rf_inputs as R
from gpu_util import FWD_TOL, GRAD_TOL, describe_mismatch, rel_l2, require_gpu, stencil_compare, to_dev, torch
from paper_2603_00035_gb300 import api

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def make_grids(count=10, seed=0, lo=17, hi=150):
    rng = np.random.default_rng(seed)
    grids = []
    for b in range(count):
        s = int(rng.integers(lo, hi + 1))
        ny, nx = (s, s) if b % 2 == 0 else (max(2, s // 2), s)
        h = 1.0 / (max(ny, nx) - 1)
        raw = R.randers_fields(ny, nx, h, 8, seed=seed * 100 + b, omega="unit", omega_scale=0.3)
        src = R.random_sources(ny, nx, int(rng.integers(1, 5)), seed=seed * 100 + b)
        g = R.sparse_loss_grad(ny, nx, 0.05, seed=b)
        grids.append(dict(raw=raw, src=src, h=h, g=g))
    return grids


@pytest.fixture(scope="module", params=["tiles", "tiled1"])
def solved(request):
    """The same grids through the tile-queue path (default) and through the
    persistent line-sweep kernel."""
    grids = make_grids()
    bs = api.BatchSolver(grids, opts=api.make_opts(variant=request.param))
    bs.run()
    torch.cuda.synchronize()
    return grids, bs, request.param


def test_batch_matches_single_grid_path(solved):
    grids, bs, variant = solved
    assert api.Context.get(0).stats()["status"] == 0
    for k, g in enumerate(grids):
        st = bs.grid(k, "status").cpu().numpy()
        assert st[0] == 0, (k, st)
        raw = to_dev(g["raw"], torch.float32)
        src = to_dev(g["src"], torch.uint8)
        proj, clip = api.rf_project(raw, 1e-6, 0.05)
        # the single-grid path with the same kernel family
        T, rec = api.rf_sweep_forward(proj, 1e-6, src, g["h"], opts=api.make_opts(variant=variant))
        sref = api.Context.get(0).stats()
        Tb = bs.grid(k, "T")
        if variant == "tiled1":
            # same schedule; only FMA contraction may differ between the kernels
            assert abs(int(st[1]) - sref["sweeps"]) <= 2, (k, st, sref)
            assert (Tb - T).abs().max().item() <= 1e-6 * T.max().item(), k
        else:
            # one queue for all grids: the rounds interleave, so the schedule
            # (not the fixed point) differs from the single-grid solve
            assert (Tb - T).abs().max().item() <= 2e-5 * T.max().item(), k
        assert (bs.grid(k, "id") == rec.id).float().mean().item() > 0.999, k
        gproj, _ = api.rf_adjoint(src, T, rec, to_dev(g["g"], torch.float32), algo="ordered")
        graw = api.rf_project_backward(raw, clip, 1e-6, 0.05, gproj)
        tol = 1e-5 if variant == "tiled1" else 1e-3
        assert rel_l2(bs.grid(k, "graw").cpu().numpy(), graw.cpu().numpy()) < tol, k


def test_batch_matches_oracle(solved):
    grids, bs, _ = solved
    for k, g in enumerate(grids[:4]):
        orc = O.solve_and_grad(g["raw"].astype(np.float64), g["src"], g["h"], 1e-6, 0.05, g["g"].astype(np.float64))
        Tb = bs.grid(k, "T").cpu().numpy()
        tmax = orc["T"].max()
        assert np.abs(Tb - orc["T"]).max() <= FWD_TOL * tmax, k
        ids = bs.grid(k, "id").cpu().numpy()
        w1 = bs.grid(k, "w1").cpu().numpy()
        flips, hard = stencil_compare(ids, w1, orc["rec"], tmax, Tb, orc["T"], fields=(orc["proj"], g["h"], 1e-6))
        assert int(hard.sum()) == 0, k
        assert rel_l2(bs.grid(k, "graw").cpu().numpy(), orc["graw"], ~flips) < GRAD_TOL, k


@pytest.mark.parametrize("variant", ["tiles", "tiled1"])
def test_batch_graph_replay_reproduces(variant):
    grids = make_grids(count=6, seed=3)
    bs = api.BatchSolver(grids, opts=api.make_opts(variant=variant))
    bs.run()
    torch.cuda.synchronize()
    T0 = bs.T.clone()
    G0 = bs.graw.clone()
    bs.capture()
    bs.T.fill_(-1.0)
    bs.graw.fill_(0.0)
    for _ in range(2):
        bs.run()
    torch.cuda.synchronize()
    assert torch.equal(bs.T, T0)
    assert torch.equal(bs.graw, G0)
    assert int(bs.gstat[:, 0].abs().sum()) == 0
    # new inputs between replays give what a run outside the graph gives
    # (a replay that reused the previous replay's multipliers would not)
    if bs.g is not None:
        bs.g.mul_(-1.5)
        graph, bs.graph = bs.graph, None
        bs.run()
        torch.cuda.synchronize()
        want = bs.graw.clone()
        bs.graph = graph
        bs.graw.fill_(0.0)
        bs.run()
        torch.cuda.synchronize()
        assert torch.equal(bs.graw, want)
        assert not torch.equal(want, G0)


@pytest.mark.parametrize("variant", ["tiles", "tiled1"])
def test_batch_grid_without_source_is_reported(variant):
    grids = make_grids(count=3, seed=5)
    grids[1]["src"] = np.zeros_like(grids[1]["src"])
    bs = api.BatchSolver(grids, opts=api.make_opts(variant=variant))
    bs.run()
    torch.cuda.synchronize()
    assert int(bs.grid(1, "status")[0]) == 6  # RF_ERR_NO_SOURCE
    assert int(bs.grid(0, "status")[0]) == 0 and int(bs.grid(2, "status")[0]) == 0
    api.Context.get(0).stats()  # clear the status word


def config3_grids(count=24, seed=0):
    """Grids of the batched workload's recipe at its sizes: long side drawn
    from 64..1024, half square and half 2:1, 1-8 sources, 8-mode fields with
    |w| = 0.3; the largest square (1024 x 1024) and the largest 2:1 grid
    (512 x 1024) are always included, and one grid has 8 sources."""
    rng = np.random.default_rng(seed)
    shapes = R.batch_shapes(count - 2, seed) + [(1024, 1024), (512, 1024)]
    grids = []
    for b, (ny, nx) in enumerate(shapes):
        h = 1.0 / (max(ny, nx) - 1)
        ns = 8 if b == len(shapes) - 1 else int(rng.integers(1, 9))
        grids.append(dict(raw=R.randers_fields(ny, nx, h, 8, seed * 1000 + b, omega="unit", omega_scale=0.3),
                          src=R.random_sources(ny, nx, ns, seed * 1000 + b),
                          g=R.sparse_loss_grad(ny, nx, 0.01, b), h=h, nsrc=ns))
    return grids


@pytest.mark.parametrize("variant", ["tiles", "tiled1"])
def test_batch_config3_sizes_match_oracle(variant):
    """rf_batch_solve at the batched workload's sizes (sides 64..1024,
    square and 2:1, 1-8 sources) against the FP64 oracle on the largest
    square grid, the largest 2:1 grid (8 sources), the smallest grid and the
    grid with the most sources: T within 1e-4 max T with identical reached
    sets, stencils equal outside near-ties, gradients within 1e-3 relative
    L2 outside the flip set."""
    grids = config3_grids()
    bs = api.BatchSolver(grids, opts=api.make_opts(variant=variant))
    bs.run()
    torch.cuda.synchronize()
    assert api.Context.get(0).stats()["status"] == 0
    assert int(bs.gstat[:, 0].abs().sum()) == 0, bs.gstat[:, 0].tolist()
    sizes = [g["src"].size for g in grids]
    nsrc = [g["nsrc"] for g in grids]
    pick = {len(grids) - 2, len(grids) - 1, int(np.argmin(sizes)),
            max(range(len(grids) - 2), key=lambda k: (nsrc[k], sizes[k]))}
    for k in sorted(pick):
        g = grids[k]
        orc = O.solve_and_grad(g["raw"].astype(np.float64), g["src"], g["h"], 1e-6, 0.05,
                               g["g"].astype(np.float64))
        To = orc["T"]
        Tb = bs.grid(k, "T").cpu().numpy()
        assert np.array_equal(np.isfinite(Tb), np.isfinite(To)), k
        fin = np.isfinite(To)
        tmax = To[fin].max()
        assert np.abs(Tb[fin] - To[fin]).max() <= FWD_TOL * tmax, (k, g["src"].shape)
        ids = bs.grid(k, "id").cpu().numpy()
        w1 = bs.grid(k, "w1").cpu().numpy()
        flips, hard = stencil_compare(ids, w1, orc["rec"], tmax, Tb, To, fields=(orc["proj"], g["h"], 1e-6))
        print(f"grid {k} {g['src'].shape} sources {g['nsrc']}: flips {flips.mean():.5f}, hard {int(hard.sum())}")
        assert int(hard.sum()) == 0, (k, g["src"].shape, describe_mismatch(hard, ids, w1, Tb, orc["rec"], To))
        assert flips.mean() <= 0.01, (k, flips.mean())
        assert rel_l2(bs.grid(k, "graw").cpu().numpy(), orc["graw"], ~flips) < GRAD_TOL, (k, g["src"].shape)


def test_batch_rejects_overlapping_descriptors():
    """Grids that overlap in the packed arrays are reported on the device
    (RF_ERR_INVALID_ARG) by the tile path."""
    import ctypes
    from paper_2603_00035_gb300 import _lib as L
    grids = make_grids(count=2, seed=7)
    bs = api.BatchSolver(grids)
    d = bs.desc.cpu().numpy().view(api._desc_dtype()).copy()
    d["offset"][1] = d["offset"][0] + 1  # second grid starts inside the first
    desc = torch.from_numpy(d.view(np.uint8)).cuda()
    crec = bs.rec.c()
    ctx = api.Context.get(0)
    L.check(L.load().rf_batch_solve(ctx.handle, ctypes.c_void_p(desc.data_ptr()), 2, int(bs.total), int(bs.max_line),
                                    ctypes.c_void_p(bs.proj.data_ptr()), 1e-6, ctypes.c_void_p(bs.src.data_ptr()),
                                    ctypes.byref(api.make_opts()), ctypes.c_void_p(bs.T.data_ptr()), ctypes.byref(crec),
                                    None, None, None, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)),
            "rf_batch_solve")
    assert ctx.stats()["status"] == L.RF_ERR_INVALID_ARG
