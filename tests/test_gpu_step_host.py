"""rf_step_host: whole steps (projection, solve, record, adjoint, projection
backward) on host buffers, pipelined across steps inside the library, against
the same kernels called one by one on device tensors (bit for bit: the same
arithmetic in the same order) and against the FP64 oracle (T; the gradients equal the device path's, which the
parity tests compare with the oracle)."""
import numpy as np
import pytest

import rf_inputs as R
from gpu_util import FWD_TOL, api, oracle_path, require_gpu, to_dev, torch
from paper_2603_00035_gb300 import _lib as L

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def device_path(c):
    raw, src, g = to_dev(c["raw"], torch.float32), to_dev(c["src"], torch.uint8), to_dev(c["g"], torch.float32)
    proj, clip = api.rf_project(raw, c["eps"], c["delta"])
    T, _ = api.rf_sweep_forward(proj, c["eps"], src, c["h"], record=False)
    rec = api.rf_record_stencils(proj, c["eps"], src, c["h"], T)
    gproj, _ = api.rf_adjoint(src, T, rec, g, algo="ordered", lam=False)
    graw = api.rf_project_backward(raw, clip, c["eps"], c["delta"], gproj)
    return T.cpu(), graw.cpu()


def test_step_host_matches_device_calls_and_oracle():
    cases = [R.config2(seed=s) for s in (0, 1, 2)]
    h = cases[0]["h"]
    pin = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a)).to(dt).pin_memory()
    raw_h = [pin(c["raw"], torch.float32) for c in cases]
    src_h = [pin(c["src"], torch.uint8) for c in cases]
    g_h = [pin(c["g"], torch.float32) for c in cases]
    T_h = [torch.empty((512, 512), dtype=torch.float32).pin_memory() for _ in cases]
    gr_h = [torch.empty((5, 512, 512), dtype=torch.float32).pin_memory() for _ in cases]
    ctx = api.Context.get(0)
    api.rf_step_host(raw_h, src_h, g_h, h, cases[0]["eps"], cases[0]["delta"], T_h, gr_h)
    assert ctx.stats()["status"] == 0
    for k, c in enumerate(cases):
        T, graw = device_path(c)
        assert torch.equal(T_h[k].view(torch.int32), T.view(torch.int32)), k
        assert torch.equal(gr_h[k].view(torch.int32), graw.view(torch.int32)), k
    orc = oracle_path(cases[1]["raw"], cases[1]["src"], h, cases[1]["eps"], cases[1]["delta"], cases[1]["g"])
    Tk = T_h[1].numpy().astype(np.float64)
    assert np.abs(Tk - orc["T"]).max() <= FWD_TOL * orc["T"].max()


def test_step_host_rejects_bad_arguments():
    c = R.config1()
    raw = torch.from_numpy(c["raw"].astype(np.float32))
    src = torch.from_numpy(c["src"])
    g = torch.from_numpy(c["g"].astype(np.float32))
    T = torch.empty((64, 64), dtype=torch.float32)
    gr = torch.empty((5, 64, 64), dtype=torch.float32)
    with pytest.raises(ValueError):
        api.rf_step_host([raw], [src], [g], c["h"], c["eps"], c["delta"], [T], [gr[:1]])
    with pytest.raises(L.RFError):  # non-positive spacing: RF_ERR_INVALID_ARG before any copy
        api.rf_step_host([raw], [src], [g], -1.0, c["eps"], c["delta"], [T], [gr])
