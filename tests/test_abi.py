"""The C-ABI library builds for sm_103a, loads without a GPU, and exports
every function include/rf.h declares.  No compute calls (no GPU here)."""
import ctypes

import pytest

from paper_2603_00035_gb300 import _lib as L
from paper_2603_00035_gb300 import build as B


@pytest.fixture(scope="module")
def lib():
    B.build()
    return L.load()


def test_header_declares_the_boundary():
    names = L.header_functions()
    for required in ("rf_project", "rf_project_backward", "rf_sweep_forward", "rf_adjoint", "rf_residual",
                     "rf_ctx_create", "rf_ctx_destroy", "rf_ctx_last_stats", "rf_status_string"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in L.header_functions():
        assert hasattr(lib, name), name


def test_status_strings(lib):
    for code, name in L.STATUS.items():
        assert lib.rf_status_string(code).decode() == name


def test_host_side_argument_checks(lib):
    # null context / null pointers are rejected on the host, before any CUDA call
    g = L.Grid(8, 8, 0.1)
    assert lib.rf_project(None, ctypes.byref(g), None, 0.0, 0.5, None, None, None) == L.RF_ERR_INVALID_ARG
    assert lib.rf_sweep_forward(None, ctypes.byref(g), None, 0.0, None, None, None, None, None) == \
        L.RF_ERR_INVALID_ARG
    assert lib.rf_adjoint(None, ctypes.byref(g), None, None, None, None, None, None, 0, None) == \
        L.RF_ERR_INVALID_ARG
    assert lib.rf_ctx_destroy(None) == L.RF_ERR_INVALID_ARG


def test_every_declared_function_has_a_signature():
    """Each function of include/rf.h gets explicit ctypes argument types (a
    float passed without them would not convert)."""
    import inspect
    from paper_2603_00035_gb300 import _lib as L
    src = inspect.getsource(L.load)
    missing = [f for f in L.header_functions() if f != "rf_status_string" and f'"{f}"' not in src]
    assert not missing, missing
