"""GB300-native AW-projection gridding and degridding (arXiv 2508.17187, Sec. 2 and Sec. 6).

The compute path is libawgrid.so (hand-written CUDA for sm_103a behind the C ABI in
include/awgrid.h); this package holds its build script and a thin Python binding.
"""
from .api import (AWG_CF_BF16, AWG_CF_FP32, AWG_DEGRID_SUBTRACT, AWG_GRID_FP64, AWG_GRID_KAHAN, CFSet, CleanWorkspace, Plan,  # noqa: F401
                  cf_set_create, cf_set_create_from_table, cf_set_load, cf_set_save, clean_hogbom, degrid_visibilities,
                  gcal_solve, grid_normalize, grid_visibilities, plan_create)
from ._lib import AwgError  # noqa: F401
