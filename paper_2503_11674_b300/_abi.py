"""ctypes declarations of the C ABI in ``include/tdp.h``.

Argument marshalling only: every computation runs in the CUDA library.  If the
library has not been built, loading it raises; there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libtdp_b300.so")

TDP_OK, TDP_ERR_INVALID, TDP_ERR_CYCLE, TDP_ERR_OOM, TDP_ERR_CUDA, TDP_ERR_STATE, TDP_ERR_TIMEOUT = range(7)
TDP_FP32, TDP_FP64 = 0, 1
STATUS_NAMES = {0: "TDP_OK", 1: "TDP_ERR_INVALID", 2: "TDP_ERR_CYCLE", 3: "TDP_ERR_OOM",
                4: "TDP_ERR_CUDA", 5: "TDP_ERR_STATE", 6: "TDP_ERR_TIMEOUT"}

# every entry point declared in include/tdp.h
EXPORTS = ["sta_build", "sta_destroy", "sta_propagate", "sta_get_timing", "sta_get_net_delays",
           "extract_critical_paths", "sta_get_paths_size", "sta_get_paths",
           "attraction_update_pairs", "attraction_reset_pairs", "attraction_set_pairs",
           "attraction_get_pairs", "attraction_loss_fwd", "attraction_loss_bwd",
           "attraction_loss_fwd_noalloc", "attraction_loss_fwd_bwd", "tdp_get_launch_count",
           "tdp_profile_kernel", "tdp_profile_read", "tdp_selftest_grid_wait", "attraction_set_loss_kind", "report_timing", "sta_join",
           "sta_propagate_incremental", "sta_incremental_stats", "net_weights_update",
           "net_weights_get", "net_weights_reset", "tdp_debug_fail_alloc",
           "tdp_debug_pending_alloc_failure", "tdp_debug_set_sync_status", "tdp_last_error"]


class NetlistDesc(C.Structure):
    _fields_ = [("n_cells", C.c_int32), ("n_pins", C.c_int32), ("n_nets", C.c_int32),
                ("pin_cell", C.c_void_p), ("net_ptr", C.c_void_p), ("pin_dir", C.c_void_p),
                ("cell_type", C.c_void_p), ("pin_dx", C.c_void_p), ("pin_dy", C.c_void_p),
                ("pin_cap", C.c_void_p), ("cell_rdrv", C.c_void_p), ("cell_fixed", C.c_void_p),
                ("r_per_um", C.c_double), ("c_per_um", C.c_double), ("d0_ps", C.c_double)]


class TdpError(RuntimeError):
    def __init__(self, fn: str, status: int, msg: str):
        super().__init__(f"{fn} -> {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None


def load() -> C.CDLL:
    """Load the library (raises FileNotFoundError if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise FileNotFoundError(
            f"{LIB_PATH} is missing: build it with `python -m paper_2503_11674_b300.build` "
            "(there is no CPU or Python fallback)")
    lib = C.CDLL(LIB_PATH)
    P, I32, I64, D = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    sig = {
        "sta_build": [C.POINTER(NetlistDesc), C.c_int, P, C.POINTER(P)],
        "sta_destroy": [P],
        "sta_propagate": [P, P, P, D, P, P],
        "sta_get_timing": [P, P, P, P],
        "sta_get_net_delays": [P, P, P, P],
        "extract_critical_paths": [P, I32, I32, I32, P],
        "sta_get_paths_size": [P, P, P, P],
        "sta_get_paths": [P, P, P, P, P, P],
        "attraction_update_pairs": [P, D, D, P],
        "attraction_reset_pairs": [P],
        "attraction_set_pairs": [P, I64, P, P],
        "attraction_get_pairs": [P, P, P, P],
        "attraction_loss_fwd": [P, P, P, D, P],
        "attraction_loss_bwd": [P, P, P, D, P, P, P],
        "attraction_loss_fwd_noalloc": [I32, P, P, P, P, P, P, P, D, P, P],
        "attraction_loss_fwd_bwd": [P, P, P, D, P, P, P, P],
        "tdp_get_launch_count": [P, P],
        "tdp_profile_kernel": [P, C.c_char_p],
        "tdp_profile_read": [P, P, P],
        "tdp_selftest_grid_wait": [C.c_double, P],
        "attraction_set_loss_kind": [P, C.c_int],
        "report_timing": [P, I32, I32, P],
        "sta_join": [P],
        "sta_propagate_incremental": [P, P, P, D, P, P],
        "sta_incremental_stats": [P, P],
        "net_weights_update": [P, D, D, P],
        "net_weights_get": [P, P],
        "net_weights_reset": [P],
        "tdp_debug_fail_alloc": [I64],
        "tdp_debug_pending_alloc_failure": [P],
        "tdp_debug_set_sync_status": [P, C.c_uint32],
        "tdp_last_error": [],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = C.c_int
    lib.sta_destroy.restype = None
    lib.tdp_last_error.restype = C.c_char_p
    _lib = lib
    return lib


def check(fn: str, status: int) -> None:
    if status != TDP_OK:
        msg = load().tdp_last_error().decode(errors="replace")
        raise TdpError(fn, status, msg)
