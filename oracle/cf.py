"""Convolution functions (CFs) of Tab. AWP-CFSETUP, built as plain FP64 DFTs (oracle).

A CF is the uv-plane kernel c_ij of Eq. CIJ (Sec. 6) for one (parallactic-angle bin,
frequency sub-band, signed w-plane).  Tab. AWP-CFSETUP builds it by convolving the
PS, A and W terms in the uv plane, which is the Fourier transform of their product
in the image plane.  Readings taken where the paper is silent:

* image-plane screen on M x M points spanning the N-pixel field, x_i = (i - M/2) N / M
  pixels, with M the smallest power of two >= max(16, 2 S) for a CF of S taps;
* screen = T(x) T(y) * A(l, m) * exp(-2 pi i w (sqrt(1 - l^2 - m^2) - 1)),
  T = psi_0(c, 2x/N) / psi_0(c, 0), c = pi W / 2, W = PS width in pixels;
* c(du, dv) = (1/M^2) sum_ij screen[j, i] exp(-2 pi i (du (i - M/2) + dv (j - M/2)) / M),
  with du, dv the sample-minus-pixel distance in grid pixels;
* tap t in [0, S) of offset o in [0, OS] sits at du = S/2 - t - o/OS, and the table is
  stored offset-major, table[oy, ox, ty, tx];
* A-term (synthetic, the paper gives no formula; parity of its physics is unpinned):
  Airy power pattern of a 25 m aperture at the sub-band frequency, elliptical by
  eps = 0.05, rotated by the parallactic angle;
* support schedule: without W every CF has `max_support` taps; with W, plane k of
  n_w planes linear in |w| over [0, w_max] has
  S_k = min(Smax, 8 ceil((8 + (Smax - 8) sqrt(k / (n_w - 1))) / 8)), at least W;
* a negative-w plane holds the CF of -|w_k|; it is built here from its own screen.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional, Sequence

import numpy as np
from scipy.special import j1

from . import pswf

C_LIGHT = 299792458.0


@dataclasses.dataclass
class CFParams:
    grid_n: int
    cell_rad: float
    oversampling: int = 20
    ps_support: int = 7
    use_ps: bool = True
    use_w: bool = False
    n_wplanes: int = 1
    w_max_lambda: float = 0.0
    use_a: bool = False
    n_pa_bins: int = 1
    pa_bin_centers: Optional[Sequence[float]] = None
    n_subbands: int = 1
    subband_freq_hz: Optional[Sequence[float]] = None
    max_support: int = 7
    dish_diameter_m: float = 25.0
    ellipticity: float = 0.05
    # full polarisation (the sparse Mueller matrix of CFs): feed squint, leakage, element cut
    use_pol: bool = False
    squint_rad: float = 0.0
    leakage: complex = 0.0
    mueller_threshold: float = 0.01

    @property
    def n_signed(self) -> int:
        return 2 * self.n_wplanes - 1 if self.use_w else 1

    @property
    def n_base(self) -> int:
        return self.n_pa_bins * self.n_subbands * self.n_signed

    @property
    def n_cf(self) -> int:
        return self.n_base * (len(mueller_elements(self)) if self.use_pol else 1)

    def cf_index(self, pa: int, sb: int, ks: int) -> int:
        return (pa * self.n_subbands + sb) * self.n_signed + ks

    def plane_w(self, ks: int) -> float:
        """w (wavelengths) of signed plane ks; ks = n_w - 1 is w = 0."""
        if not self.use_w:
            return 0.0
        k = ks - (self.n_wplanes - 1)
        return k * self.w_max_lambda / (self.n_wplanes - 1)


def support_of_plane(p: CFParams, ks: int) -> int:
    if not p.use_w:
        return int(p.max_support)
    k = abs(ks - (p.n_wplanes - 1))
    q = math.sqrt(k / (p.n_wplanes - 1))
    s = 8 * math.ceil((8.0 + (p.max_support - 8) * q) / 8.0)
    s = min(s, p.max_support)
    return max(s, p.ps_support)


def supports(p: CFParams) -> np.ndarray:
    out = np.zeros(p.n_cf, dtype=np.int32)
    for e in range(p.n_cf // p.n_base):
        for pa in range(p.n_pa_bins):
            for sb in range(p.n_subbands):
                for ks in range(p.n_signed):
                    out[e * p.n_base + p.cf_index(pa, sb, ks)] = support_of_plane(p, ks)
    return out


# Polarisation products in the order RR, RL, LR, LL: product k correlates feed k // 2 of the first
# antenna with feed k % 2 of the second (R = 0, L = 1).
def mueller_elements(p: CFParams):
    """Kept Mueller elements (p, q), row-major: the element of output product p = (a, b) and sky
    product q = (c, d) carries |d|^n with n = [a != c] + [b != d] leakage factors; it is kept when
    that is at least the threshold (reading of Sec. 6, where the sparse Mueller matrix of CFs keeps
    only the elements that matter at the instrument's sensitivity)."""
    dmag = abs(complex(p.leakage))
    out = []
    for pp in range(4):
        for qq in range(4):
            n = (pp // 2 != qq // 2) + (pp % 2 != qq % 2)
            if n == 0 or dmag ** n >= p.mueller_threshold:
                out.append((pp, qq))
    return out


def airy_voltage(rho_rad, freq_hz: float, dish_m: float) -> np.ndarray:
    x = math.pi * dish_m * np.asarray(rho_rad) * freq_hz / C_LIGHT
    out = np.ones_like(x)
    nz = x != 0
    out[nz] = 2.0 * j1(x[nz]) / x[nz]
    return out


def screen_size(S: int) -> int:
    M = 16
    while M < 2 * S:
        M *= 2
    return M


def airy_power(rho_rad, freq_hz: float, dish_m: float) -> np.ndarray:
    x = math.pi * dish_m * np.asarray(rho_rad) * freq_hz / C_LIGHT
    out = np.ones_like(x)
    nz = x != 0
    out[nz] = (2.0 * j1(x[nz]) / x[nz]) ** 2
    return out


def screen(p: CFParams, pa: int, sb: int, ks: int, M: int, elem=None) -> np.ndarray:
    """Image-plane product of the enabled terms, complex128 [M(y), M(x)].  With a Mueller element
    elem = (p, q) the A factor is J_ac conj(J_bd) for p = (a, b), q = (c, d), from the Jones matrix
    J = [[A_R, d A_R], [d A_L, A_L]] of voltage patterns squinted by -+squint along the rotated l
    axis (the outer product of the two antennas' Jones matrices, Sec. 2, evaluated in the image
    plane; reading: a synthetic feed model, the paper gives none)."""
    i = np.arange(M, dtype=np.float64)
    x = (i - M / 2) * p.grid_n / M                  # image pixels from the field centre
    lm = x * p.cell_rad                             # direction cosines
    if p.use_ps:
        t1 = pswf.taper(p.ps_support, 2.0 * x / p.grid_n)
    else:
        t1 = np.ones(M)
    s = (t1[:, None] * t1[None, :]).astype(np.complex128)
    L = lm[None, :]
    Mm = lm[:, None]
    if p.use_w:
        w = p.plane_w(ks)
        s = s * np.exp(-2j * math.pi * w * (np.sqrt(1.0 - L * L - Mm * Mm) - 1.0))
    if p.use_a:
        chi = float(p.pa_bin_centers[pa])
        lr = L * math.cos(chi) + Mm * math.sin(chi)
        mr = -L * math.sin(chi) + Mm * math.cos(chi)
        eps = p.ellipticity
        nu = float(p.subband_freq_hz[sb])
        if elem is None:
            rho = np.sqrt((lr / (1.0 + eps)) ** 2 + (mr / (1.0 - eps)) ** 2)
            s = s * airy_power(rho, nu, p.dish_diameter_m)
        else:
            rho_r = np.sqrt(((lr - p.squint_rad) / (1.0 + eps)) ** 2 + (mr / (1.0 - eps)) ** 2)
            rho_l = np.sqrt(((lr + p.squint_rad) / (1.0 + eps)) ** 2 + (mr / (1.0 - eps)) ** 2)
            ar = airy_voltage(rho_r, nu, p.dish_diameter_m)
            al = airy_voltage(rho_l, nu, p.dish_diameter_m)
            d = complex(p.leakage)
            J = [[ar + 0j, d * ar], [d * al, al + 0j]]
            pp, qq = elem
            a, b, c, e = pp // 2, pp % 2, qq // 2, qq % 2
            s = s * (J[a][c] * np.conj(J[b][e]))
    return s


def tap_positions(S: int, OS: int) -> np.ndarray:
    """du[o, t] = S/2 - t - o/OS: sample-minus-pixel distance of tap t at offset o."""
    o = np.arange(OS + 1, dtype=np.float64)[:, None]
    t = np.arange(S, dtype=np.float64)[None, :]
    return S / 2.0 - t - o / OS


def cf_table(p: CFParams, pa: int, sb: int, ks: int, elem=None) -> np.ndarray:
    """complex128 [OS+1, OS+1, S, S] table of one CF (offset-major)."""
    S = support_of_plane(p, ks)
    OS = p.oversampling
    M = screen_size(S)
    s = screen(p, pa, sb, ks, M, elem)
    d = tap_positions(S, OS).reshape(-1)                     # Q = (OS+1) S
    i = np.arange(M, dtype=np.float64) - M / 2
    E = np.exp(-2j * math.pi * np.outer(d, i) / M) / M       # [Q, M]
    full = E @ s @ E.T                                        # [Q(v), Q(u)]
    return full.reshape(OS + 1, S, OS + 1, S).transpose(0, 2, 1, 3).copy()


def cf_set(p: CFParams, which: Optional[Sequence[int]] = None):
    """All (or the listed) CF tables: dict cf_index -> table.  A full-polarisation set holds one
    block of n_base CFs per kept Mueller element, element e at e * n_base + cf_index."""
    out = {}
    elems = mueller_elements(p) if p.use_pol else [None]
    for e, el in enumerate(elems):
        for pa in range(p.n_pa_bins):
            for sb in range(p.n_subbands):
                for ks in range(p.n_signed):
                    ci = e * p.n_base + p.cf_index(pa, sb, ks)
                    if which is None or ci in which:
                        out[ci] = cf_table(p, pa, sb, ks, el)
    return out


def flatten_cf_set(p: CFParams, tables: dict):
    """Concatenate tables into one complex128 buffer with per-CF offsets (in elements)."""
    sup = supports(p)
    offs = np.zeros(p.n_cf + 1, dtype=np.int64)
    per = (p.oversampling + 1) ** 2 * sup.astype(np.int64) ** 2
    offs[1:] = np.cumsum(per)
    buf = np.zeros(int(offs[-1]), dtype=np.complex128)
    for ci, t in tables.items():
        buf[offs[ci]:offs[ci + 1]] = t.reshape(-1)
    return buf, offs[:-1].copy(), sup
