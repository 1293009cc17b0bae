"""Grid <-> image transforms, taper correction and brute-force DFT references (oracle, FP64).

* ``grid_to_image``: F-dagger of Eq. IMAGE-MOD on an N x N grid whose uv origin is pixel
  N/2, giving the image whose phase centre is pixel N/2:
  image[j] = sum_g grid[g] exp(+2 pi i (g - N/2)(j - N/2) / N) per axis.
* ``image_to_grid``: F of Eq. ME-MOD-GRIDDED, the same sum with exp(-2 pi i ...).
* ``dirty_image``: Re(F-dagger G) / (sum of weights * T(l) T(m)), T the PS taper, so that
  a point of flux S peaks at S (Eq. IMAGE-MOD with the Sec. 6 PS term divided out).
* ``dft_dirty_image``: the same image by direct summation over samples,
  I(l, m) = sum_s w_s Re(V_s exp(+2 pi i (u l + v m + w (n - 1)))) / sum_s w_s.
* ``point_source_vis``: V(u, v, w) = sum_k S_k exp(-2 pi i (u l_k + v m_k + w (n_k - 1)))
  (Eq. ME with a sky of point sources, no Mueller terms).
"""
from __future__ import annotations

import math

import numpy as np

from . import pswf

C_LIGHT = 299792458.0


def grid_to_image(grid_c: np.ndarray) -> np.ndarray:
    """F-dagger over axes (0, 1) of [N, N, ...] with both origins at N/2 (no normalisation)."""
    N = grid_c.shape[0]
    g = np.fft.ifftshift(grid_c, axes=(0, 1))
    im = np.fft.ifft2(g, axes=(0, 1)) * (N * N)
    return np.fft.fftshift(im, axes=(0, 1))


def image_to_grid(image: np.ndarray) -> np.ndarray:
    """F over axes (0, 1) of [N, N, ...] with both origins at N/2 (no normalisation)."""
    im = np.fft.ifftshift(image, axes=(0, 1))
    g = np.fft.fft2(im, axes=(0, 1))
    return np.fft.fftshift(g, axes=(0, 1))


def taper_image(N: int, ps_support: int) -> np.ndarray:
    """T(x) for image pixels x = j - N/2, j in [0, N)."""
    x = (np.arange(N) - N // 2).astype(np.float64)
    return pswf.taper(ps_support, 2.0 * x / N)


def dirty_image(grid_c: np.ndarray, sumwt, ps_support: int, use_ps: bool = True) -> np.ndarray:
    """Re(F-dagger grid) / (sumwt * T T): float64 [N, N, P]."""
    N = grid_c.shape[0]
    im = grid_to_image(grid_c).real
    t = taper_image(N, ps_support) if use_ps else np.ones(N)
    corr = t[:, None] * t[None, :]
    return im / (np.asarray(sumwt)[None, None, :] * corr[:, :, None])


def model_to_grid(model: np.ndarray, ps_support: int, use_ps: bool = True) -> np.ndarray:
    """F of model / (T T) for degridding a model image [N, N, P] (taper divided out first)."""
    N = model.shape[0]
    t = taper_image(N, ps_support) if use_ps else np.ones(N)
    corr = t[:, None] * t[None, :]
    return image_to_grid(model / corr[:, :, None])


def dft_dirty_image(uvw_m, freq_hz, vis, weight, N: int, cell: float, pix_y, pix_x,
                    with_w: bool = True) -> np.ndarray:
    """Brute-force dirty image at the listed pixels (vis, weight: [R, C] single pol).

    with_w=False drops the w (n - 1) phase: the image that plain 2-D gridding approximates.
    """
    pix_y = np.asarray(pix_y)
    pix_x = np.asarray(pix_x)
    l = (pix_x - N // 2) * cell
    m = (pix_y - N // 2) * cell
    nm1 = np.sqrt(1.0 - l * l - m * m) - 1.0
    if not with_w:
        nm1 = np.zeros_like(nm1)
    out = np.zeros(l.shape[0])
    sw = 0.0
    for c in range(freq_hz.shape[0]):
        sc = freq_hz[c] / C_LIGHT
        u, v, w = uvw_m[:, 0] * sc, uvw_m[:, 1] * sc, uvw_m[:, 2] * sc
        wv = weight[:, c] * vis[:, c]
        ph = np.outer(u, l) + np.outer(v, m) + np.outer(w, nm1)
        out += (wv[:, None] * np.exp(2j * math.pi * ph)).real.sum(axis=0)
        sw += weight[:, c].sum()
    return out / sw


def point_source_vis(uvw_m, freq_hz, l, m, flux) -> np.ndarray:
    """complex128 [R, C] visibilities of point sources at (l, m) with the given fluxes."""
    nm1 = np.sqrt(1.0 - l * l - m * m) - 1.0
    out = np.zeros((uvw_m.shape[0], freq_hz.shape[0]), dtype=np.complex128)
    for c in range(freq_hz.shape[0]):
        sc = freq_hz[c] / C_LIGHT
        ph = (np.outer(uvw_m[:, 0] * sc, l) + np.outer(uvw_m[:, 1] * sc, m)
              + np.outer(uvw_m[:, 2] * sc, nm1))
        out[:, c] = (flux[None, :] * np.exp(-2j * math.pi * ph)).sum(axis=1)
    return out
