"""ctypes binding of librf (include/rf.h).  Marshalling only: every step of
the solver runs in the CUDA library; if librf.so cannot be loaded this
module raises -- there is no fallback."""
from __future__ import annotations

import ctypes
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
HEADER = os.path.join(ROOT, "include", "rf.h")
LIB_PATH = os.path.join(HERE, "librf.so")

STATUS = {0: "RF_OK", 1: "RF_ERR_INVALID_ARG", 2: "RF_ERR_CUDA", 3: "RF_ERR_NOT_CONVERGED",
          4: "RF_ERR_TIMEOUT", 5: "RF_ERR_NONFINITE_INPUT", 6: "RF_ERR_NO_SOURCE",
          7: "RF_ERR_NO_MEMORY", 8: "RF_ERR_UNSUPPORTED"}
RF_OK, RF_ERR_INVALID_ARG, RF_ERR_CUDA, RF_ERR_NOT_CONVERGED, RF_ERR_TIMEOUT = 0, 1, 2, 3, 4
RF_ERR_NONFINITE_INPUT, RF_ERR_NO_SOURCE, RF_ERR_NO_MEMORY, RF_ERR_UNSUPPORTED = 5, 6, 7, 8
RF_SWEEP_AUTO, RF_SWEEP_TILED1, RF_SWEEP_STREAMED, RF_SWEEP_TILED4, RF_SWEEP_TILES = 0, 1, 2, 4, 8
RF_MODE_COLD, RF_MODE_WARM = 0, 1
RF_ADJ_SWEEP, RF_ADJ_ORDERED, RF_ADJ_LEVELS, RF_ADJ_TILES = 0, 1, 2, 3


class RFError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)}")


class Grid(ctypes.Structure):
    _fields_ = [("ny", ctypes.c_int32), ("nx", ctypes.c_int32), ("h", ctypes.c_float)]


class Opts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_float), ("max_sweeps", ctypes.c_int32), ("mode", ctypes.c_int32),
                ("band", ctypes.c_int32), ("block", ctypes.c_int32), ("rtol", ctypes.c_float),
                ("variant", ctypes.c_int32), ("window", ctypes.c_float)]


class MetricParams(ctypes.Structure):
    _fields_ = [("lam_min", ctypes.c_float), ("lam_max", ctypes.c_float), ("b_max", ctypes.c_float),
                ("delta", ctypes.c_float), ("eps", ctypes.c_float)]


RF_TV_NONE, RF_TV_FROBENIUS, RF_TV_LOG_EUCLIDEAN = 0, 1, 2


class Record(ctypes.Structure):
    _fields_ = [("id", ctypes.c_void_p), ("w1", ctypes.c_void_p), ("dT", ctypes.c_void_p)]


class BatchDesc(ctypes.Structure):
    _fields_ = [("ny", ctypes.c_int32), ("nx", ctypes.c_int32), ("h", ctypes.c_float), ("pad", ctypes.c_int32),
                ("offset", ctypes.c_int64)]


class Stats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("sweeps", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("adj_sweeps", ctypes.c_int32), ("cell_updates", ctypes.c_int64),
                ("max_residual", ctypes.c_float), ("rounds", ctypes.c_int32)]


_lib = None


def header_functions():
    """Names of the functions include/rf.h declares."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rf_[a-z_0-9]+)\s*\(", text)))


def load(path: str = LIB_PATH):
    """Load librf.so (built by paper_2603_00035_gb300.build); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"librf.so not found at {path}: run paper_2603_00035_gb300.build.build() "
                           "(the CUDA library is required; there is no CPU fallback)")
    lib = ctypes.CDLL(path)
    P, I, F = ctypes.c_void_p, ctypes.c_int, ctypes.c_float
    sig = {
        "rf_ctx_create": [ctypes.POINTER(P), I],
        "rf_ctx_destroy": [P],
        "rf_ctx_set_timeout": [P, ctypes.c_int64],
        "rf_ctx_set_adjoint_park": [P, ctypes.c_int64],
        "rf_ctx_last_stats": [P, ctypes.POINTER(Stats)],
        "rf_project": [P, ctypes.POINTER(Grid), P, F, F, P, P, P],
        "rf_project_backward": [P, ctypes.POINTER(Grid), P, P, F, F, P, P, P],
        "rf_sweep_forward": [P, ctypes.POINTER(Grid), P, F, P, ctypes.POINTER(Opts), P,
                             ctypes.POINTER(Record), P],
        "rf_residual": [P, ctypes.POINTER(Grid), P, F, P, P, P, P, P],
        "rf_record_stencils": [P, ctypes.POINTER(Grid), P, F, P, P, ctypes.POINTER(Record), P],
        "rf_adjoint": [P, ctypes.POINTER(Grid), P, P, ctypes.POINTER(Record), P, P, P, I, P],
        "rf_batch_solve": [P, P, I, ctypes.c_int64, ctypes.c_int32, P, F, P, ctypes.POINTER(Opts), P,
                           ctypes.POINTER(Record), P, P, P, P],
        "rf_sweep_forward_static": [ctypes.POINTER(Grid), P, F, P, ctypes.POINTER(Opts), P,
                                    ctypes.POINTER(Stats), P],
        "rf_metric_project": [P, ctypes.POINTER(Grid), P, ctypes.POINTER(MetricParams), P, P, P],
        "rf_metric_project_backward": [P, ctypes.POINTER(Grid), P, ctypes.POINTER(MetricParams), P, P, P, P],
        "rf_tv": [P, ctypes.POINTER(Grid), P, I, F, F, P, P, P],
        "rf_encoder_combine": [P, P, I, I, I, I, P, I, F, P, P],
        "rf_encoder_combine_backward": [P, P, I, I, I, I, I, F, P, P, P],
        "rf_softmin_forward": [P, ctypes.POINTER(Grid), P, F, P, F, ctypes.POINTER(Opts), P, P],
        "rf_softmin_record": [P, ctypes.POINTER(Grid), P, F, P, P, F, P, P, P],
        "rf_softmin_adjoint": [P, ctypes.POINTER(Grid), P, P, P, P, P, P, P, P],
    }
    I64 = ctypes.c_int64
    sig.update({
        "rf_unet_conv3x3": [P, P, I, I, I, I, P, P, I, I, P, P, P],
        "rf_unet_conv3x3_tc": [P, P, I, I, I, I, P, P, I, I, P, P, P],
        "rf_unet_conv3x3_wgrad": [P, P, P, I, I, I, I, I, P, P],
        "rf_unet_conv3x3_wgrad_tc": [P, P, P, I, I, I, I, I, P, P],
        "rf_step_host": [P, ctypes.POINTER(Grid), I, P, P, P, F, F, ctypes.POINTER(Opts), I, P, P, P],
        "rf_unet_bias_grad": [P, P, I64, I, P, P],
        "rf_unet_flip_weights": [P, P, I, I, P, P],
        "rf_unet_maxpool2": [P, P, I, I, I, I, P, P, P],
        "rf_unet_maxpool2_backward": [P, P, P, I, I, I, I, P, P],
        "rf_unet_upsample2": [P, P, I, I, I, I, P, P],
        "rf_unet_upsample2_backward": [P, P, I, I, I, I, P, P],
        "rf_unet_concat": [P, P, I, P, I, I64, P, I, P],
        "rf_unet_relu_backward": [P, P, P, I64, P],
        "rf_unet_mse": [P, P, I, P, P, I64, F, P, P, P],
        "rf_unet_cast_bf16": [P, P, P, I64, P],
        "rf_unet_pack_input": [P, P, I, I, I, I, I, P, P],
        "rf_unet_add": [P, P, P, I64, P],
        "rf_unet_source_features": [P, I, I, I, F, P, P, P, P],
        "rf_unet_box_down": [P, P, I, I, I, I, P, P],
        "rf_unet_bilinear": [P, P, I, I, I, I, I, F, P, P],
    })
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    lib.rf_status_string.argtypes = [I]
    lib.rf_status_string.restype = ctypes.c_char_p
    _lib = lib
    return lib


def check(status: int, where: str):
    if status != RF_OK:
        raise RFError(status, where)
