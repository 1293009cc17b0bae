"""Shared test helpers: one workload description feeds both the oracle and the library."""
from __future__ import annotations

import numpy as np

from oracle import cf as ocf


def oracle_params(wl, **over) -> ocf.CFParams:
    p = dict(grid_n=wl.grid_n, cell_rad=wl.cell_rad, oversampling=wl.oversampling, ps_support=wl.ps_support,
             use_w=wl.use_w, n_wplanes=wl.n_wplanes, w_max_lambda=wl.w_max_lambda, use_a=wl.use_a,
             n_pa_bins=wl.n_pa_bins, pa_bin_centers=list(wl.pa_bin_centers), n_subbands=wl.n_subbands,
             subband_freq_hz=list(wl.subband_freq_hz), max_support=wl.max_support)
    p.update(over)
    return ocf.CFParams(**p)


def library_params(op: ocf.CFParams, cf_dtype: int = 0, separable: bool = True) -> dict:
    return dict(grid_n=op.grid_n, cell_rad=op.cell_rad, oversampling=op.oversampling, ps_support=op.ps_support,
                use_ps=op.use_ps, use_w=op.use_w, n_wplanes=op.n_wplanes, w_max_lambda=op.w_max_lambda,
                use_a=op.use_a, n_pa_bins=op.n_pa_bins,
                pa_bin_centers_rad=(np.asarray(op.pa_bin_centers, dtype=np.float64) if op.pa_bin_centers is not None else None),
                n_subbands=op.n_subbands,
                subband_freq_hz=(np.asarray(op.subband_freq_hz, dtype=np.float64) if op.subband_freq_hz is not None else None),
                max_support=op.max_support, dish_diameter_m=op.dish_diameter_m, ellipticity=op.ellipticity,
                cf_dtype=cf_dtype, separable=separable, use_pol=op.use_pol, squint_rad=op.squint_rad,
                leakage=complex(op.leakage), mueller_threshold=op.mueller_threshold)


def rel_rms(a, b) -> float:
    a = np.asarray(a)
    b = np.asarray(b)
    den = np.sqrt(np.sum(np.abs(b) ** 2))
    return float(np.sqrt(np.sum(np.abs(a - b) ** 2)) / den) if den > 0 else float(np.sqrt(np.sum(np.abs(a) ** 2)))


def inner_half(img):
    """Central N/2 x N/2 of an [N, N, ...] image: the region where the PS taper is >= 0.25.

    Outside it the taper correction divides by T(x) T(y) down to ~1e-7 at the corners, which
    magnifies any FP32 rounding by up to 1e7; dirty-image errors are gated on this region.
    """
    N = img.shape[0]
    return img[N // 4:3 * N // 4, N // 4:3 * N // 4]


def mosaic_row_phase(wl, seed=4) -> np.ndarray:
    """Per-row (dl, dm) of a two-field mosaic: pointings on alternating integrations, +-30 / +-20
    cells from the image centre, plus a per-row jitter of up to 2 cells (the mean pointing offset of
    the row's two antennas).  float64 [R, 2]."""
    rng = np.random.default_rng(seed)
    R = wl.n_rows
    field = (np.arange(R) // wl.n_bl) % 2
    dl = np.where(field == 0, 30.0, -30.0) * wl.cell_rad
    dm = np.where(field == 0, -20.0, 20.0) * wl.cell_rad
    jit = rng.uniform(-2.0, 2.0, (R, 2)) * wl.cell_rad
    return np.stack([dl + jit[:, 0], dm + jit[:, 1]], -1)
