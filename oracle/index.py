"""Per-sample index rules (oracle, FP64): uv scaling, w-plane, CF, pixel and offset.

Eq. CIJ (Sec. 6) selects the kernel CF_ij(nu, w, t) per visibility; Eq. Appendix-IMEQ
sums over nu and w.  The paper does not fix the discretisation; the reading used:

* u_lambda = u_m * (nu / c) for every (row, channel), in FP64;
* x = u_lambda * (N * cell) + N/2 (grid pixel; the uv origin is pixel N/2), same for y;
* with W on, k = floor(|w_lambda| * (n_w - 1) / w_max + 1/2); k > n_w - 1 drops the
  sample; the signed plane is ks = n_w - 1 + k for w >= 0 and n_w - 1 - k for w < 0;
* cf = (pa_bin * n_sb + subband) * n_signed + ks, S = its tap count;
* hx = x - S/2, first tap p0x = floor(hx) + 1, fraction fx = p0x - hx in (0, 1],
  offset ox = floor(fx * OS + 1/2) in [0, OS]; same for y;
* the sample is kept iff -1 <= hx < N - S and -1 <= hy < N - S (every tap on the grid);
* optional phase-centre shift (dl, dm): phasor exp(+2 pi i (u dl + v dm + w dn)),
  dn = sqrt(1 - dl^2 - dm^2) - 1 (the phase-gradient term of Eq. CIJ).

Every step is a separate IEEE FP64 operation (numpy never fuses multiply-add), so the
integer results are reproducible bit for bit by any implementation of the same steps.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

from .cf import CFParams, supports as cf_supports

C_LIGHT = 299792458.0


@dataclasses.dataclass
class SampleIndex:
    valid: np.ndarray   # bool  [R*C]
    cf: np.ndarray      # int32 [R*C]
    p0x: np.ndarray     # int64 [R*C]
    p0y: np.ndarray
    ox: np.ndarray      # int32 [R*C]
    oy: np.ndarray
    support: np.ndarray  # int32 [R*C]
    phasor: Optional[np.ndarray] = None   # complex128 [R*C] or None


def sample_index(p: CFParams, uvw_m, freq_hz, pa_bin=None, chan_subband=None,
                 phase_shift=None, supports=None, row_phase=None) -> SampleIndex:
    """Index every (row, channel) sample; `supports` overrides the schedule (caller-made tables).

    Phase term of Eq. CIJ (reading: exp(+2 pi i u.(s_0 - s(P) - (Delta s_i + Delta s_j)/2)) with the
    offset of the image centre from the phase centre, w included through dn = sqrt(1 - dl^2 - dm^2)
    - 1): `phase_shift` (dl, dm) applies to every row; `row_phase` [R, 2] gives each row its own
    (dl, dm) - the pointing of a mosaic field and the mean pointing offset of the row's antennas
    (Tab. AWPSETUP-MOSAICKING) - and replaces `phase_shift`."""
    uvw_m = np.asarray(uvw_m, dtype=np.float64)
    freq_hz = np.asarray(freq_hz, dtype=np.float64)
    R, C = uvw_m.shape[0], freq_hz.shape[0]
    sc = freq_hz / C_LIGHT
    u = uvw_m[:, 0:1] * sc[None, :]
    v = uvw_m[:, 1:2] * sc[None, :]
    w = uvw_m[:, 2:3] * sc[None, :]
    N = p.grid_n
    scale = float(N) * p.cell_rad
    half = float(N // 2)
    x = u * scale + half
    y = v * scale + half
    valid = np.isfinite(x) & np.isfinite(y)
    if p.use_w:
        inv_dw = float(p.n_wplanes - 1) / p.w_max_lambda
        t = np.abs(w) * inv_dw
        k = np.floor(t + 0.5)
        valid &= np.isfinite(k) & (k <= p.n_wplanes - 1)
        k = np.where(valid, k, 0).astype(np.int64)
        ks = (p.n_wplanes - 1) + np.where(w < 0, -k, k)
    else:
        ks = np.zeros((R, C), dtype=np.int64)
    pa = np.zeros((R, 1), dtype=np.int64) if p.n_pa_bins == 1 else np.asarray(pa_bin, dtype=np.int64)[:, None]
    sb = np.zeros((1, C), dtype=np.int64) if p.n_subbands == 1 else np.asarray(chan_subband, dtype=np.int64)[None, :]
    cf = (pa * p.n_subbands + sb) * p.n_signed + ks
    sup_tab = cf_supports(p) if supports is None else np.asarray(supports, dtype=np.int32)
    S = sup_tab[cf].astype(np.float64)
    hx = x - S * 0.5
    hy = y - S * 0.5
    valid &= (hx >= -1.0) & (hx < N - S) & (hy >= -1.0) & (hy < N - S)
    hx = np.where(valid, hx, 0.0)
    hy = np.where(valid, hy, 0.0)
    p0x = np.floor(hx) + 1.0
    p0y = np.floor(hy) + 1.0
    fx = p0x - hx
    fy = p0y - hy
    OS = float(p.oversampling)
    ox = np.floor(fx * OS + 0.5)
    oy = np.floor(fy * OS + 0.5)
    ph = None
    if row_phase is not None:
        rp = np.asarray(row_phase, dtype=np.float64)
        dl, dm = rp[:, 0:1], rp[:, 1:2]
        dn = np.sqrt(1.0 - dl * dl - dm * dm) - 1.0
        turns = u * dl + v * dm + w * dn
        ph = np.exp(2j * math.pi * turns).reshape(-1)
    elif phase_shift is not None:
        dl, dm = float(phase_shift[0]), float(phase_shift[1])
        dn = math.sqrt(1.0 - dl * dl - dm * dm) - 1.0
        turns = u * dl + v * dm + w * dn
        ph = np.exp(2j * math.pi * turns).reshape(-1)
    return SampleIndex(valid=valid.reshape(-1), cf=cf.reshape(-1).astype(np.int32),
                       p0x=p0x.reshape(-1).astype(np.int64), p0y=p0y.reshape(-1).astype(np.int64),
                       ox=ox.reshape(-1).astype(np.int32), oy=oy.reshape(-1).astype(np.int32),
                       support=sup_tab[cf].reshape(-1).astype(np.int32), phasor=ph)
