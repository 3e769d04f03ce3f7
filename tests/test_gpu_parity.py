"""GPU (CUDA, through the C ABI) vs FP64 oracle parity on seeded inputs.

Sizes: the 64x64 and 512x512 workloads, a ragged multi-source grid that
spans several bands and blocks with partial tails, and degenerate shapes.
"""
import numpy as np
import pytest

import rf_inputs as R
from gpu_util import (FWD_TOL, GRAD_TOL, api, canonical_stencil, describe_mismatch, flip_mask, gpu_path,
                      oracle_path, rel_l2, require_gpu, stencil_compare, to_dev, torch)
import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def ragged_case():
    ny, nx = 203, 141  # several bands/blocks with partial tails
    h = 1.0 / 202
    return dict(raw=R.randers_fields(ny, nx, h, 8, seed=9, omega="field", omega_max=1.0),
                src=R.random_sources(ny, nx, 3, seed=9), h=h, eps=1e-6, delta=0.3,
                g=R.sparse_loss_grad(ny, nx, 0.05, seed=9))


CASES = {"config1": R.config1, "ragged": ragged_case, "config2": R.config2}


@pytest.fixture(scope="module", params=list(CASES))
def case(request):
    c = CASES[request.param]()
    gpu = gpu_path(c["raw"], c["src"], c["h"], c["eps"], c["delta"], c["g"])
    orc = oracle_path(c["raw"], c["src"], c["h"], c["eps"], c["delta"], c["g"])
    return request.param, c, gpu, orc


def test_projection_parity(case):
    name, c, gpu, orc = case
    same = gpu["clip"] == orc["clip"]
    assert same.mean() > 0.999
    assert np.allclose(gpu["proj"][:, same], orc["proj"][:, same], rtol=2e-6, atol=1e-7)


def test_forward_parity(case):
    name, c, gpu, orc = case
    assert gpu["st_fwd"]["status"] == 0, gpu["st_fwd"]
    assert gpu["st_fwd"]["converged"]
    Tg, To = gpu["T"], orc["T"]
    assert np.array_equal(np.isfinite(Tg), np.isfinite(To))
    fin = np.isfinite(To)
    tmax = To[fin].max()
    err = np.abs(Tg[fin] - To[fin]).max()
    assert err <= FWD_TOL * tmax, (name, err, tmax)
    assert np.all(Tg[c["src"] == 1] == 0.0)


# bound on the fraction of nodes whose (canonical) stencil differs from the
# oracle's -- all of them near-ties -- per workload
FLIP_BOUND = {"config1": 0.01, "ragged": 0.01, "config2": 0.01}


def test_record_parity(case):
    name, c, gpu, orc = case
    T = orc["T"]
    tmax = T[np.isfinite(T)].max()
    flips, hard = stencil_compare(gpu["rec_np"]["id"], gpu["rec_np"]["w1"], orc["rec"], tmax, gpu["T"], T,
                                  fields=(orc["proj"], c["h"], c["eps"]))
    raw_diff = gpu["rec_np"]["id"] != orc["rec"]["id"]
    print(f"{name}: ids differ {raw_diff.mean():.4f}, canonical flips {flips.mean():.5f} "
          f"({int(flips.sum())} nodes), hard mismatches {int(hard.sum())}")
    # near-ties (oracle margin < 1e-5 max T) may pick either stencil; outside
    # them the GPU must name the oracle's stencil
    assert int(hard.sum()) == 0, (name, describe_mismatch(hard, gpu["rec_np"]["id"], gpu["rec_np"]["w1"], gpu["T"],
                                                           orc["rec"], T))
    assert flips.mean() <= FLIP_BOUND[name], (name, flips.mean())
    keep = ~flips
    _, w_g = canonical_stencil(gpu["rec_np"]["id"], gpu["rec_np"]["w1"], with_weight=True)
    _, w_o = canonical_stencil(orc["rec"]["id"], orc["rec"]["w1"], with_weight=True)
    bad = keep & ~np.isclose(w_g, w_o, atol=2e-3, rtol=0.0)
    assert not bad.any(), (name, int(bad.sum()), describe_mismatch(bad, gpu["rec_np"]["id"], gpu["rec_np"]["w1"],
                                                                  gpu["T"], orc["rec"], T))
    dTg, dTo = gpu["rec_np"]["dT"], orc["rec"]["dT"]
    assert rel_l2(dTg, dTo, keep) < GRAD_TOL


def test_gradient_parity(case):
    name, c, gpu, orc = case
    assert gpu["st_adj"]["status"] == 0, gpu["st_adj"]
    flips, _ = flip_mask(gpu, orc)
    keep = ~flips
    e_lam = rel_l2(gpu["lam"], orc["lam"], keep)
    e_proj = rel_l2(gpu["gproj"], orc["gproj"], keep)
    e_raw = rel_l2(gpu["graw"], orc["graw"], keep)
    assert e_proj < GRAD_TOL and e_raw < GRAD_TOL, (name, e_lam, e_proj, e_raw, flips.sum())


def test_ordered_adjoint_matches_sweep_and_oracle(case):
    """RF_ADJ_ORDERED (radix sort on T + dependency-ordered gather) on the
    GPU record: same lambda as the transposed-sweep adjoint up to float32
    summation order, and within the gradient tolerance of the oracle."""
    name, c, gpu, orc = case
    src = to_dev(c["src"], torch.uint8)
    T = to_dev(gpu["T"], torch.float32)
    g = to_dev(c["g"], torch.float32)
    gproj, lam = api.rf_adjoint(src, T, gpu["rec"], g, algo="ordered")
    st = api.Context.get(0).stats()
    assert st["status"] == 0, st
    lam, gproj = lam.cpu().numpy(), gproj.cpu().numpy()
    assert rel_l2(lam, gpu["lam"]) < 1e-5
    assert rel_l2(gproj, gpu["gproj"]) < 1e-5
    flips, _ = flip_mask(gpu, orc)
    assert rel_l2(gproj, orc["gproj"], ~flips) < GRAD_TOL


@pytest.mark.parametrize("algo", ["sweep", "ordered", "tiles"])
def test_adjoint_kernel_on_oracle_record(algo):
    """The adjoint kernel alone, fed the oracle's record (cast to float32):
    lambda and the contracted gradients must match the FP64 back-substitution
    to float32 accuracy."""
    c = R.config1()
    orc = oracle_path(c["raw"], c["src"], c["h"], c["eps"], c["delta"], c["g"])
    rec = api.Record(to_dev(orc["rec"]["id"], torch.uint8), to_dev(orc["rec"]["w1"], torch.float32),
                     to_dev(orc["rec"]["dT"], torch.float32))
    T = to_dev(orc["T"], torch.float32)
    src = to_dev(c["src"], torch.uint8)
    g = to_dev(np.where(np.isfinite(orc["T"]), c["g"], 0.0), torch.float32)
    gproj, lam = api.rf_adjoint(src, T, rec, g, algo=algo)
    st = api.Context.get(0).stats()
    assert st["status"] == 0
    assert rel_l2(lam.cpu().numpy(), orc["lam"]) < 1e-5
    assert rel_l2(gproj.cpu().numpy(), orc["gproj"]) < 1e-5


def test_residual_of_gpu_solution_is_small():
    c = R.config2()
    raw = to_dev(c["raw"], torch.float32)
    src = to_dev(c["src"], torch.uint8)
    proj, _ = api.rf_project(raw, c["eps"], c["delta"])
    T, _ = api.rf_sweep_forward(proj, c["eps"], src, c["h"], record=False)
    mx = api.rf_residual(proj, c["eps"], src, c["h"], T)
    tmax = T.max().item()
    assert mx.item() <= 1e-6 * tmax
    # independent check in FP64 at sampled nodes with the oracle's candidate set
    Tn = T.cpu().numpy().astype(np.float64)
    pr = proj.cpu().numpy().astype(np.float64)
    res = O.residual(pr, c["src"], c["h"], c["eps"], Tn)
    assert np.abs(res).max() <= 2e-6 * tmax


@pytest.mark.parametrize("shape", [(1, 57), (57, 1), (2, 2), (33, 65), (130, 7)])
def test_degenerate_shapes(shape):
    ny, nx = shape
    h = 0.1
    raw = R.randers_fields(ny, nx, h, 4, seed=1, omega="unit", omega_scale=0.2)
    src = R.point_sources(ny, nx, [(ny // 2, nx // 2)])
    prj, _ = O.project(raw, 1e-6, 0.05)
    To, _, _, _ = O.solve_gs(prj, src, h, 1e-6)
    proj, _ = api.rf_project(to_dev(raw, torch.float32), 1e-6, 0.05)
    T, _ = api.rf_sweep_forward(proj, 1e-6, to_dev(src, torch.uint8), h)
    st = api.Context.get(0).stats()
    assert st["status"] == 0 and st["converged"]
    assert np.abs(T.cpu().numpy() - To).max() <= FWD_TOL * To.max()


def test_no_source_and_all_sources():
    ny, nx = 40, 50
    raw = to_dev(R.randers_fields(ny, nx, 0.1, 4, seed=2), torch.float32)
    proj, _ = api.rf_project(raw, 1e-6, 0.05)
    ctx = api.Context.get(0)
    T, _ = api.rf_sweep_forward(proj, 1e-6, torch.zeros((ny, nx), dtype=torch.uint8, device="cuda"), 0.1)
    st = ctx.stats()
    assert st["status"] == 6  # RF_ERR_NO_SOURCE
    assert torch.isinf(T).all()
    T, rec = api.rf_sweep_forward(proj, 1e-6, torch.ones((ny, nx), dtype=torch.uint8, device="cuda"), 0.1)
    st = ctx.stats()
    assert st["status"] == 0 and (T == 0).all() and (rec.id == 0).all()


def test_nonfinite_input_is_reported():
    ny, nx = 16, 16
    raw = R.randers_fields(ny, nx, 0.1, 4, seed=2)
    raw[3, 5, 5] = np.nan
    api.rf_project(to_dev(raw, torch.float32), 1e-6, 0.05)
    assert api.Context.get(0).stats()["status"] == 5  # RF_ERR_NONFINITE_INPUT


def test_timeout_path_returns_cleanly():
    """A zero wait bound makes the first unsatisfied device wait expire: the
    launch must end with RF_ERR_TIMEOUT and leave the context usable."""
    c = R.config2()
    raw = to_dev(c["raw"], torch.float32)
    src = to_dev(c["src"], torch.uint8)
    ctx = api.Context(0)
    proj, _ = api.rf_project(raw, c["eps"], c["delta"], ctx=ctx)
    ctx.set_timeout(0)
    api.rf_sweep_forward(proj, c["eps"], src, c["h"], record=False, ctx=ctx)
    st = ctx.stats()
    assert st["status"] == 4  # RF_ERR_TIMEOUT
    ctx.set_timeout(2_000_000_000)
    T, rec = api.rf_sweep_forward(proj, c["eps"], src, c["h"], ctx=ctx)
    st = ctx.stats()
    assert st["status"] == 0 and st["converged"]
    g = to_dev(c["g"], torch.float32)
    for algo in ("sweep", "ordered", "tiles"):
        ctx.set_timeout(0)
        api.rf_adjoint(src, T, rec, g, algo=algo, ctx=ctx)
        assert ctx.stats()["status"] == 4, algo  # RF_ERR_TIMEOUT
        ctx.set_timeout(2_000_000_000)
        api.rf_adjoint(src, T, rec, g, algo=algo, ctx=ctx)
        assert ctx.stats()["status"] == 0, algo


@pytest.mark.parametrize("band,block,variant", [(32, 8, 4), (64, 32, 4), (128, 16, 4), (16, 16, 4), (32, 32, 1),
                                               (16, 16, 1), (64, 16, 1), (24, 4, 1), (128, 32, 1), (32, 32, 2),
                                               (64, 16, 2), (32, 16, 2), (16, 16, 2), (8, 4, 2)])
def test_band_and_block_shapes_agree(band, block, variant):
    c = ragged_case()
    prj, _ = O.project(c["raw"], c["eps"], c["delta"])
    To, _, _, _ = O.solve_gs(prj, c["src"], c["h"], c["eps"])
    proj, _ = api.rf_project(to_dev(c["raw"], torch.float32), c["eps"], c["delta"])
    T, _ = api.rf_sweep_forward(proj, c["eps"], to_dev(c["src"], torch.uint8), c["h"],
                                opts=api.make_opts(band=band, block=block, variant=variant), record=False)
    st = api.Context.get(0).stats()
    assert st["status"] == 0 and st["converged"]
    assert np.abs(T.cpu().numpy() - To).max() <= FWD_TOL * To.max()


@pytest.mark.parametrize("which", ["config1", "config2"])
def test_sweep_variants_agree(which):
    """The kernel variants evaluate the same 16 candidates per node (the
    streamed one in the cone form); only FP32 rounding differs, so T agrees
    to a few ulp and the reached sets are identical."""
    c = CASES[which]()
    proj, _ = api.rf_project(to_dev(c["raw"], torch.float32), c["eps"], c["delta"])
    src = to_dev(c["src"], torch.uint8)
    out = {}
    for v in ("tiled1", "tiled4", "streamed", "tiles"):
        out[v], _ = api.rf_sweep_forward(proj, c["eps"], src, c["h"], opts=api.make_opts(variant=v), record=False)
        st = api.Context.get(0).stats()
        assert st["status"] == 0 and st["converged"], v
    for v in ("tiled1", "streamed", "tiles"):
        assert torch.equal(torch.isfinite(out[v]), torch.isfinite(out["tiled4"])), v
        assert (out[v] - out["tiled4"]).abs().max().item() <= 1e-5 * out["tiled4"].max().item(), v


@pytest.mark.parametrize("which", ["config1", "config2"])
def test_bitwise_change_test_still_converges_here(which):
    """tol = rtol = 0 (stop only at a sweep with no bitwise change) proves a
    fixed point when it terminates; on these workloads it does, and agrees
    with the default relative test."""
    c = CASES[which]()
    proj, _ = api.rf_project(to_dev(c["raw"], torch.float32), c["eps"], c["delta"])
    src = to_dev(c["src"], torch.uint8)
    T0, _ = api.rf_sweep_forward(proj, c["eps"], src, c["h"], opts=api.make_opts(rtol=0.0), record=False)
    st = api.Context.get(0).stats()
    assert st["status"] == 0 and st["converged"]
    T1, _ = api.rf_sweep_forward(proj, c["eps"], src, c["h"], record=False)
    assert api.Context.get(0).stats()["status"] == 0
    assert (T0 - T1).abs().max().item() <= 1e-5 * T0.max().item()


@pytest.mark.parametrize("variant", ["streamed", "tiled1", "tiled4", "tiles"])
def test_table1_isotropic_refinement_on_gpu(variant):
    """The CUDA path on the paper's isotropic refinement study (Table 1,
    fixture tests/golden/table1_isotropic.txt): errors against the exact
    distance within 10 % of the printed values (3 % from 100^2 up), and T
    within FP32 rounding of the FP64 oracle."""
    import os
    rows = []
    for line in open(os.path.join(os.path.dirname(__file__), "golden", "table1_isotropic.txt")):
        line = line.strip()
        if line and not line.startswith("#"):
            n, h, l2, linf = line.split()
            rows.append((int(n), float(h), float(l2), float(linf)))
    for n, h, l2_ref, linf_ref in rows:
        raw = np.zeros((5, n, n), np.float32)
        raw[0] = raw[2] = 1.0
        src = np.zeros((n, n), np.uint8)
        c = n // 2
        src[c, c] = 1
        proj, _ = api.rf_project(to_dev(raw, torch.float32), 0.0, 0.05)
        T, _ = api.rf_sweep_forward(proj, 0.0, to_dev(src, torch.uint8), h, opts=api.make_opts(variant=variant),
                                    record=False)
        st = api.Context.get(0).stats()
        assert st["status"] == 0 and st["converged"], (n, st)
        Tg = T.cpu().numpy().astype(np.float64)
        y, x = np.mgrid[0:n, 0:n] * h
        err = Tg - np.hypot(x - c * h, y - c * h)
        l2, linf = float(np.sqrt(np.mean(err ** 2))), float(np.abs(err).max())
        tol = 0.10 if n < 100 else 0.03
        assert abs(l2 - l2_ref) <= tol * l2_ref, (n, l2, l2_ref)
        assert abs(linf - linf_ref) <= tol * linf_ref, (n, linf, linf_ref)
        prj, _ = O.project(raw.astype(np.float64), 0.0, 0.05)
        To, _, _, _ = O.solve_gs(prj, src, h, 0.0)
        assert np.abs(Tg - To).max() <= FWD_TOL * To.max(), n



@pytest.mark.parametrize("window", [0.25, 1.0, 2.0, 8.0, 1e9])
def test_tile_queue_windows_agree(window):
    """The tile queue reaches the oracle's fixed point whatever its
    delta-stepping window (a window of 1e9 processes every queued tile in
    every round)."""
    c = ragged_case()
    prj, _ = O.project(c["raw"], c["eps"], c["delta"])
    To, _, _, _ = O.solve_gs(prj, c["src"], c["h"], c["eps"])
    proj, _ = api.rf_project(to_dev(c["raw"], torch.float32), c["eps"], c["delta"])
    T, _ = api.rf_sweep_forward(proj, c["eps"], to_dev(c["src"], torch.uint8), c["h"],
                                opts=api.make_opts(variant="tiles", window=window), record=False)
    st = api.Context.get(0).stats()
    assert st["status"] == 0 and st["converged"], st
    assert st["rounds"] > 0
    Tg = T.cpu().numpy()
    assert np.array_equal(np.isfinite(Tg), np.isfinite(To))
    assert np.abs(Tg - To).max() <= FWD_TOL * To.max()


def test_tile_queue_is_deterministic():
    """Tiles read their neighbours' state as of the round's start, so two
    solves give bitwise-identical T whatever order the CTAs take tiles in."""
    c = R.config2()
    proj, _ = api.rf_project(to_dev(c["raw"], torch.float32), c["eps"], c["delta"])
    src = to_dev(c["src"], torch.uint8)
    outs = []
    for _ in range(3):
        T, _ = api.rf_sweep_forward(proj, c["eps"], src, c["h"], opts=api.make_opts(variant="tiles"), record=False)
        assert api.Context.get(0).stats()["status"] == 0
        outs.append(T.clone())
    assert torch.equal(outs[0], outs[1]) and torch.equal(outs[0], outs[2])


@pytest.mark.parametrize("shape,src_ij", [((40, 33), (20, 32)), ((33, 33), (32, 32)), ((65, 97), (0, 64)),
                                          ((64, 64), (31, 32))])
def test_tile_queue_sources_on_tile_edges(shape, src_ij):
    """Sources on a tile edge or alone in a one-column / one-node edge tile:
    the tiles across the edge must still be reached."""
    ny, nx = shape
    h = 1.0 / (max(ny, nx) - 1)
    raw = R.randers_fields(ny, nx, h, 4, seed=4, omega="unit", omega_scale=0.3)
    src = R.point_sources(ny, nx, [src_ij])
    prj, _ = O.project(raw, 1e-6, 0.05)
    To, _, _, _ = O.solve_gs(prj, src, h, 1e-6)
    proj, _ = api.rf_project(to_dev(raw, torch.float32), 1e-6, 0.05)
    T, _ = api.rf_sweep_forward(proj, 1e-6, to_dev(src, torch.uint8), h, opts=api.make_opts(variant="tiles"),
                                record=False)
    st = api.Context.get(0).stats()
    assert st["status"] == 0 and st["converged"], st
    Tg = T.cpu().numpy()
    assert np.isfinite(Tg).all()
    assert np.abs(Tg - To).max() <= FWD_TOL * To.max()
