"""Hogbom CLEAN, the minor cycle of the imaging loop (Sec. 5.2: the model update of Eq. ModelUpdate
with point components), written out as its textbook steps.

TEST INFRASTRUCTURE ONLY (see the package header).

The search decides integer pixel positions from floating-point values, so this restatement works
in the precision of the GPU minor cycle, IEEE FP32, with every product and difference rounded
separately (numpy float32 arithmetic); the pixel choice then agrees exactly.  Reading taken where
the paper is silent: the component is the pixel of largest |residual| in the search window, ties
going to the lowest row-major index; the loop stops for good once that value is below the
threshold; the PSF (peak at (Np/2, Np/2)) is subtracted wherever its shifted copy overlaps the
image.
"""
from __future__ import annotations

import numpy as np


def hogbom(residual: np.ndarray, psf: np.ndarray, n_iter: int, gain: float, threshold: float = 0.0,
           window=None):
    """Return (residual, model, components) after at most n_iter Hogbom iterations (float32)."""
    res = np.array(residual, dtype=np.float32, copy=True)
    N = res.shape[0]
    model = np.zeros_like(res)
    psf = np.asarray(psf, dtype=np.float32)
    Np = psf.shape[0]
    x0, x1, y0, y1 = (0, N, 0, N) if window is None else window
    gain32 = np.float32(gain)
    comps = []
    for _ in range(n_iter):
        sub = np.abs(res[y0:y1, x0:x1])
        k = int(np.argmax(sub))               # first occurrence: the lowest row-major index
        py, px = y0 + k // (x1 - x0), x0 + k % (x1 - x0)
        if not sub.flat[k] >= np.float32(threshold):
            break
        g = np.float32(gain32 * res[py, px])
        model[py, px] = np.float32(model[py, px] + g)
        comps.append((py, px, float(g)))
        # residual[y][x] -= g * psf[y - py + Np/2][x - px + Np/2] where that PSF pixel exists
        ya, yb = max(0, py - Np // 2), min(N, py - Np // 2 + Np)
        xa, xb = max(0, px - Np // 2), min(N, px - Np // 2 + Np)
        patch = psf[ya - py + Np // 2:yb - py + Np // 2, xa - px + Np // 2:xb - px + Np // 2]
        res[ya:yb, xa:xb] = res[ya:yb, xa:xb] - (g * patch).astype(np.float32)
    return res, model, comps
