"""Learned warm start: the batched training-data solver, the replacement
(non-min) warm update, and a trained network's warm start, all judged
against the cold solve and the residual check."""
import numpy as np
import pytest

import oracle as O
import rf_inputs as R
from gpu_util import FWD_TOL, require_gpu, to_dev, torch
from paper_2603_00035_gb300 import api, warmstart as WS

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def test_batch_forward_matches_single_grid():
    x, T, gstat = WS.make_samples([11, 12, 13], n=64)
    assert int(gstat[:, 0].abs().sum()) == 0
    assert x.shape == (3, 64, 64, 16) and x.dtype == torch.bfloat16
    from rf_inputs import gpu as G
    h = 1.0 / 63
    for b, seed in enumerate([11, 12, 13]):
        raw = G.randers_fields_batch([seed], 64, h, 8 if seed % 2 == 0 else 16)[0].contiguous()
        src, _ = G.random_sources_batch([seed], 64)
        proj, _ = api.rf_project(raw, 1e-6, 0.05)
        Tr, _ = api.rf_sweep_forward(proj, 1e-6, src[0].contiguous(), h, record=False)
        # the batch shares one tile queue across its grids: same fixed point,
        # another schedule than the single-grid solve
        assert (T[b] - Tr).abs().max().item() <= 2e-5 * Tr.max().item()


@pytest.mark.parametrize("scale,which", [(0.5, "config1"), (1.3, "config2")])
def test_replacement_update_recovers_from_bad_guesses(scale, which):
    """Warm starts from a guess below (0.5 T) or above (1.3 T) the solution
    reach the cold solution: an underestimate cannot freeze in (it rises
    about one edge cost per sweep, so the underestimate case uses the small
    grid and a larger sweep cap)."""
    c = R.config1() if which == "config1" else R.config2()
    proj, _ = api.rf_project(to_dev(c["raw"], torch.float32), c["eps"], c["delta"])
    src = to_dev(c["src"], torch.uint8)
    Tc, _ = api.rf_sweep_forward(proj, c["eps"], src, c["h"], record=False)
    T0 = (Tc * scale).contiguous()
    Tw, _ = api.rf_sweep_forward(proj, c["eps"], src, c["h"], opts=api.make_opts(warm=True, max_sweeps=1000),
                                 T=T0, record=False)
    st = api.Context.get(0).stats()
    assert st["status"] == 0 and st["converged"], st
    assert (Tw - Tc).abs().max().item() <= FWD_TOL * Tc.max().item()


def test_trained_network_warm_start_is_correct_and_measured():
    """Train briefly on solver-generated samples, warm-start a 1024^2 solve,
    and check it against the cold solve and the residual test.  The sweep
    counts of both are printed: that is the measured gain (it may be small:
    the sweep count is set by how often characteristics turn)."""
    net, tr = WS.train(samples=128, chunk=64, batch=8)
    assert tr["loss_history"][-1] < tr["loss_history"][0]
    n = 1024
    h = 1.0 / (n - 1)
    raw = torch.from_numpy(R.randers_fields(n, n, h, 16, 77, omega="unit", omega_scale=0.3)).cuda()
    src = torch.from_numpy(R.random_sources(n, n, 3, 77)).cuda()
    proj, _ = api.rf_project(raw, 1e-6, 0.05)
    Tc, _ = api.rf_sweep_forward(proj, 1e-6, src, h, record=False)
    stc = api.Context.get(0).stats()
    Tw, info = WS.solve(net, raw, src, h)
    assert (Tw - Tc).abs().max().item() <= FWD_TOL * Tc.max().item()
    assert info["residual"] <= 1e-5 * Tc.max().item() or info["fallback"]
    print(f"cold sweeps {stc['sweeps']}, warm sweeps {info['warm_sweeps']}, fallback {info['fallback']}")


def test_warm_solve_without_fallback_matches_oracle():
    """A warm-started 1024^2 solve from the network's resampled guess, run to
    its own fixed point (sweep cap high enough that the cold fallback never
    fires), against the FP64 oracle: identical reached set and max |dT| <=
    1e-4 max T."""
    net, _ = WS.train(samples=64, chunk=64, batch=8)
    n = 1024
    h = 1.0 / (n - 1)
    raw_np = R.randers_fields(n, n, h, 16, 78, omega="unit", omega_scale=0.3)
    src_np = R.random_sources(n, n, 2, 78)
    Tw, info = WS.solve(net, torch.from_numpy(raw_np).cuda(), torch.from_numpy(src_np).cuda(), h,
                        opts=api.make_opts(max_sweeps=1000))
    assert not info["fallback"], info
    prj, _ = O.project(raw_np.astype(np.float64), 1e-6, 0.05)
    To, _, st, _ = O.solve_gs(prj, src_np, h, 1e-6)
    assert st == O.OK
    Tw = Tw.cpu().numpy()
    assert np.array_equal(np.isfinite(Tw), np.isfinite(To))
    fin = np.isfinite(To)
    err = np.abs(Tw[fin] - To[fin]).max()
    print(f"warm 1024^2: sweeps {info['warm_sweeps']}, max |dT| / max T = {err / To[fin].max():.2e}")
    assert err <= FWD_TOL * To[fin].max()


def test_warm_and_cold_time_to_accuracy_measured():
    """Cold and warm starts of a 1024^2 solve with the tile queue.  The
    exact runs (rtol 1e-6) end within 1e-4 max T of the cold solution -- the
    same accuracy -- and their time ratio is measured and printed (a briefly
    trained network: the ratio is whatever it is; the test pins that it is
    measured and finite).  The runs with a 1e-4 stopping tolerance are
    printed too: such a tolerance lets changes below it stop propagating, so
    it does not deliver 1e-4 accuracy (its error is reported, not bounded)."""
    net, _ = WS.train(samples=64, chunk=64, batch=8)
    n = 1024
    h = 1.0 / (n - 1)
    raw = torch.from_numpy(R.randers_fields(n, n, h, 16, 79, omega="unit", omega_scale=0.3)).cuda()
    src = torch.from_numpy(R.random_sources(n, n, 3, 79)).cuda()
    rows = WS.compare(net, raw, src, h)
    for name, r in rows.items():
        if name == "guess":
            continue
        assert r["status"] == "RF_OK", (name, r)
        assert np.isfinite(r["err"]), (name, r)
        if name.endswith("exact"):
            assert r["err"] <= FWD_TOL, (name, r)
    ratio = (rows["warm_exact"]["ms"] + rows["guess"]["ms"]) / rows["cold_exact"]["ms"]
    print(f"1024^2 at 1e-4 accuracy: cold {rows['cold_exact']['ms']:.2f} ms, warm {rows['warm_exact']['ms']:.2f} ms "
          f"+ guess {rows['guess']['ms']:.2f} ms: warm/cold {ratio:.2f}; 1e-4 stopping tolerance: cold err "
          f"{rows['cold_loose']['err']:.1e}, warm err {rows['warm_loose']['err']:.1e}")
    assert 0.0 < ratio < 1e3
