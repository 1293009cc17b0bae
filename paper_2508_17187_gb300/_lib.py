"""ctypes view of the awgrid C ABI (include/awgrid.h).  Marshalling only: every computation runs
in libawgrid.so.  Importing this module never builds or falls back; a missing library raises."""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libawgrid.so")

AWG_OK = 0
STATUS_NAMES = {0: "AWG_OK", 1: "AWG_ERR_INVALID_ARG", 2: "AWG_ERR_UNSUPPORTED", 3: "AWG_ERR_OOM",
                4: "AWG_ERR_CUDA", 5: "AWG_ERR_TIMEOUT"}
AWG_CF_FP32, AWG_CF_BF16 = 0, 1
AWG_GRID_KAHAN, AWG_GRID_FP64 = 1, 2
AWG_DEGRID_SUBTRACT = 1

EXPORTED = ["cf_set_create", "cf_set_create_from_table", "cf_set_destroy", "cf_set_info", "cf_set_fused_terms", "cf_set_get_params", "cf_set_save", "cf_set_load",
            "cf_set_get_supports",
            "cf_set_copy_table", "cf_set_copy_factors", "plan_create", "plan_update", "plan_destroy", "plan_stats", "plan_check", "plan_copy_index", "grid_visibilities",
            "degrid_visibilities", "grid_normalize", "awg_last_error", "awg_kernel_launches",
            "grid_visibilities_noalloc", "grid_visibilities_plain_fp64", "degrid_visibilities_plain_fp64",
            "awg_fp32_fma_probe", "awg_fp64_fma_probe", "cf_set_autotune", "cf_set_choose", "clean_hogbom_workspace_bytes",
            "clean_hogbom", "clean_hogbom_components", "plan_set_row_phase", "gcal_workspace_bytes", "gcal_solve",
            "cf_set_mueller", "awg_debug_fail_allocations", "awg_debug_live_allocations", "awg_debug_ws_withhold"]


class AwgError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        self.status = status
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")


class CfParams(ctypes.Structure):
    _fields_ = [
        ("grid_n", ctypes.c_int),
        ("cell_rad", ctypes.c_double),
        ("oversampling", ctypes.c_int),
        ("ps_support", ctypes.c_int),
        ("use_ps", ctypes.c_int),
        ("use_w", ctypes.c_int),
        ("n_wplanes", ctypes.c_int),
        ("w_max_lambda", ctypes.c_double),
        ("use_a", ctypes.c_int),
        ("n_pa_bins", ctypes.c_int),
        ("pa_bin_centers_rad", ctypes.POINTER(ctypes.c_double)),
        ("n_subbands", ctypes.c_int),
        ("subband_freq_hz", ctypes.POINTER(ctypes.c_double)),
        ("max_support", ctypes.c_int),
        ("dish_diameter_m", ctypes.c_double),
        ("ellipticity", ctypes.c_double),
        ("cf_dtype", ctypes.c_int),
        ("separable", ctypes.c_int),
        ("use_pol", ctypes.c_int),
        ("squint_rad", ctypes.c_double),
        ("leakage_re", ctypes.c_double),
        ("leakage_im", ctypes.c_double),
        ("mueller_threshold", ctypes.c_double),
    ]


_lock = threading.Lock()
_lib = None


def load():
    """Load the in-tree libawgrid.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2508_17187_gb300.build.build() "
                               "(there is no fallback implementation)")
        lib = ctypes.CDLL(LIB_PATH)
        vp, i32, i64, f64p = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.POINTER(ctypes.c_double)
        st = ctypes.c_int
        sig = {
            "cf_set_create": ([ctypes.POINTER(CfParams), vp, ctypes.POINTER(vp)], st),
            "cf_set_create_from_table": ([ctypes.POINTER(CfParams), vp, vp, vp, ctypes.POINTER(vp)], st),
            "cf_set_destroy": ([vp], st),
            "cf_set_info": ([vp, ctypes.POINTER(i32), ctypes.POINTER(i64), ctypes.POINTER(i32)], st),
            "cf_set_fused_terms": ([vp, ctypes.POINTER(i32)], st),
            "cf_set_get_params": ([vp, ctypes.POINTER(CfParams), vp, vp], st),
            "cf_set_save": ([vp, ctypes.c_char_p], st),
            "cf_set_load": ([ctypes.c_char_p, vp, ctypes.POINTER(vp)], st),
            "cf_set_get_supports": ([vp, vp], st),
            "cf_set_copy_table": ([vp, i32, vp], st),
            "cf_set_copy_factors": ([vp, i32, i32, vp, vp, vp], st),
            "plan_create": ([vp, vp, i64, vp, i32, vp, vp, vp, vp, ctypes.POINTER(vp)], st),
            "plan_update": ([vp, vp, vp, vp, vp, vp], st),
            "plan_destroy": ([vp], st),
            "plan_stats": ([vp, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i64)], st),
            "plan_copy_index": ([vp, vp, vp, vp, vp, vp, vp], st),
            "plan_check": ([vp], st),
            "grid_visibilities": ([vp, vp, vp, vp, i32, vp, vp, vp, i32, vp], st),
            "degrid_visibilities": ([vp, vp, vp, vp, i32, i32, vp], st),
            "grid_normalize": ([vp, vp, i32, vp, i32, vp], st),
            "awg_last_error": ([], ctypes.c_char_p),
            "awg_kernel_launches": ([], ctypes.c_int64),
            "grid_visibilities_noalloc": ([vp, vp, i64, vp, i32, vp, vp, vp, vp, i32, vp, vp, vp], st),
            "grid_visibilities_plain_fp64": ([vp, vp, i64, vp, i32, i32, i32, vp, vp, vp, vp, i32, vp, vp, vp], st),
            "degrid_visibilities_plain_fp64": ([vp, vp, i64, vp, i32, i32, i32, vp, vp, vp, vp, i32, vp], st),
            "awg_fp32_fma_probe": ([vp, i32, i64, vp, ctypes.POINTER(ctypes.c_double)], st),
            "awg_fp64_fma_probe": ([vp, i32, i64, vp, ctypes.POINTER(ctypes.c_double)], st),
            "cf_set_autotune": ([vp, vp, i64, vp, i32, vp, vp, i32, vp, vp, vp], st),
            "cf_set_choose": ([vp, i32, i32], st),
            "clean_hogbom_workspace_bytes": ([], ctypes.c_int64),
            "clean_hogbom": ([vp, vp, i32, vp, i32, i32, ctypes.c_float, ctypes.c_float, vp, vp, vp], st),
            "clean_hogbom_components": ([vp, ctypes.POINTER(ctypes.c_int32)], st),
            "plan_set_row_phase": ([vp, vp, vp, vp, vp], st),
            "gcal_workspace_bytes": ([i64, i32, i32, i32, i32, i32], ctypes.c_int64),
            "cf_set_mueller": ([vp, vp, vp, vp], st),
            "awg_debug_fail_allocations": ([ctypes.c_int64], st),
            "awg_debug_live_allocations": ([], ctypes.c_int64),
            "awg_debug_ws_withhold": ([ctypes.c_int32], st),
            "gcal_solve": ([vp, vp, vp, i64, i32, i32, i32, vp, vp, i32, i32, i32, ctypes.c_double, ctypes.c_double,
                            i32, i32, vp, vp, vp, vp], st),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


def check(status: int, where: str):
    if status != AWG_OK:
        msg = load().awg_last_error()
        raise AwgError(status, where, msg.decode() if msg else "")
