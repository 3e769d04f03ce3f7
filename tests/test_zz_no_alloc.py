"""rf_sweep_forward_static: the forward solve for callers that cannot
allocate device memory at solve time (a host framework that already owns the
device's memory or enforces a budget, or a loop that must not pay
cudaMalloc's device-wide synchronisation).  Its scratch is a fixed
file-scope device array inside librf, so the call itself allocates nothing.

The test calls it through the C ABI twice in a row and compares each result
with the allocating rf_sweep_forward on the same inputs, within the forward
tolerance used by the other parity tests.  Nothing here depends on earlier
tests, so it passes alone in a fresh process or after the rest of the suite.
"""
import ctypes

import numpy as np
import pytest

import rf_inputs as R
from gpu_util import FWD_TOL, api, require_gpu, to_dev, torch
from paper_2603_00035_gb300 import _lib as L

pytestmark = pytest.mark.gpu


def _static_fn():
    lib = L.load()
    fn = lib.rf_sweep_forward_static
    fn.argtypes = [ctypes.POINTER(L.Grid), ctypes.c_void_p, ctypes.c_float, ctypes.c_void_p,
                   ctypes.POINTER(L.Opts), ctypes.c_void_p, ctypes.POINTER(L.Stats), ctypes.c_void_p]
    fn.restype = ctypes.c_int
    return fn


def test_static_entry_matches_allocating_entry_twice():
    require_gpu()
    fn = _static_fn()
    c = R.config2()  # 512 x 512 = 262144 nodes, within the 1048576-node limit
    ny, nx = c["src"].shape
    raw = to_dev(c["raw"], torch.float32)
    src = to_dev(c["src"], torch.uint8)
    proj, _ = api.rf_project(raw, c["eps"], c["delta"])
    # the entry without allocation runs the tiled kernel (the streamed one
    # needs a record buffer)
    T_ref, _ = api.rf_sweep_forward(proj, c["eps"], src, c["h"], opts=api.make_opts(variant="tiled1"), record=False)
    st_ref = api.Context.get(0).stats()
    assert st_ref["status"] == 0 and st_ref["converged"]
    tmax = T_ref.max().item()
    grid = L.Grid(ny, nx, c["h"])
    opts = api.make_opts()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        T = torch.full((ny, nx), float("nan"), dtype=torch.float32, device="cuda")
        st = L.Stats()
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        status = fn(ctypes.byref(grid), ctypes.c_void_p(proj.data_ptr()), c["eps"],
                    ctypes.c_void_p(src.data_ptr()), ctypes.byref(opts), ctypes.c_void_p(T.data_ptr()),
                    ctypes.byref(st), stream)
        assert status == L.RF_OK, (call, L.STATUS.get(status, status))
        if call == 1:  # the first call may load the module; the second must not allocate anything
            assert torch.cuda.mem_get_info()[0] == free_before, "the call allocated device memory"
        assert st.converged == 1 and st.sweeps == st_ref["sweeps"], (call, st.sweeps, st_ref["sweeps"])
        err = (T - T_ref).abs().max().item()
        assert err <= FWD_TOL * tmax, (call, err)


def test_static_entry_rejects_oversized_grids():
    require_gpu()
    fn = _static_fn()
    grid = L.Grid(1025, 1024, 0.001)  # 1049600 nodes > 1048576
    opts = api.make_opts()
    dummy = torch.zeros(8, device="cuda")
    p = ctypes.c_void_p(dummy.data_ptr())
    st = L.Stats()
    assert fn(ctypes.byref(grid), p, 1e-6, p, ctypes.byref(opts), p, ctypes.byref(st), None) == \
        L.RF_ERR_INVALID_ARG
    grid = L.Grid(64, 64, 0.01)
    opts = api.make_opts(max_sweeps=5000)  # beyond the 1024-sweep limit
    assert fn(ctypes.byref(grid), p, 1e-6, p, ctypes.byref(opts), p, ctypes.byref(st), None) == \
        L.RF_ERR_INVALID_ARG


def test_static_entry_warm_mode_asynchronous():
    """Warm mode with stats = NULL (the asynchronous path): start from 1.2 x
    the allocating entry's solution, synchronise, and compare."""
    require_gpu()
    fn = _static_fn()
    c = R.config1()
    ny, nx = c["src"].shape
    proj, _ = api.rf_project(to_dev(c["raw"], torch.float32), c["eps"], c["delta"])
    src = to_dev(c["src"], torch.uint8)
    T_ref, _ = api.rf_sweep_forward(proj, c["eps"], src, c["h"], opts=api.make_opts(variant="tiled1"), record=False)
    assert api.Context.get(0).stats()["status"] == 0
    T = (T_ref * 1.2).contiguous()
    grid = L.Grid(ny, nx, c["h"])
    opts = api.make_opts(warm=True, max_sweeps=256)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    status = fn(ctypes.byref(grid), ctypes.c_void_p(proj.data_ptr()), c["eps"], ctypes.c_void_p(src.data_ptr()),
                ctypes.byref(opts), ctypes.c_void_p(T.data_ptr()), None, stream)
    assert status == L.RF_OK, L.STATUS.get(status, status)
    torch.cuda.synchronize()
    assert (T - T_ref).abs().max().item() <= FWD_TOL * T_ref.max().item()
