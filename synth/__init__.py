"""Seeded synthetic VLA-shaped inputs shared by the oracle tests, the GPU tests and the bench.

This module only makes inputs: antenna layout, uvw tracks, channel frequencies,
point-source skies, noise and natural weights.  It holds none of the resampling
arithmetic (index rules, convolution functions, gridding, degridding, tapers); the
oracle and the CUDA library each implement those on their own.

The shapes follow the paper's deployment example (Sec. 6: VLA A-array, S band,
2-4 GHz, wide-band W/AW-projection imaging).  The archival data set is not
available, so these generators stand in for it:

* array: 27 antennas on a Y (3 arms 120 deg apart, rotated 5 deg from north),
  9 per arm at radii 21 km * (k/9)**1.716, +-0.5 % seeded jitter, latitude 34.08 deg;
* track: declination -27.8 deg, hour angle -3 h .. +3 h split evenly over the
  integrations; rows are time-major (row = t * n_baselines + b);
* sky: point sources, flux U(0.1, 1) Jy; exact visibilities
  sum_k S_k exp(-2 pi i (u l_k + v m_k + w (n_k - 1))) with the phase in FP64;
* noise: complex Gaussian, sigma = 1 mJy per part, jittered x U(0.8, 1.2) per
  baseline, natural weights 1/sigma^2;
* pols RR, RL, LR, LL: sky in RR/LL, noise only in RL/LR.

Seeds: layout 20250817, noise 1, sky 2, finite-difference directions 3.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

C_LIGHT = 299792458.0
LAT_DEG = 34.08
DEC_DEG = -27.8
SEED_LAYOUT = 20250817
SEED_NOISE = 1
SEED_SKY = 2
SEED_FD = 3


def antenna_enu(seed: int = SEED_LAYOUT) -> np.ndarray:
    """27 antenna positions (east, north, up) in metres on a VLA-like Y."""
    rng = np.random.default_rng(seed)
    pos = []
    for arm in range(3):
        theta = math.radians(5.0 + 120.0 * arm)
        for k in range(1, 10):
            r = 21000.0 * (k / 9.0) ** 1.716 * (1.0 + rng.uniform(-0.005, 0.005))
            pos.append((r * math.sin(theta), r * math.cos(theta), 0.0))
    return np.asarray(pos, dtype=np.float64)


def baselines_xyz(enu: np.ndarray, lat_deg: float = LAT_DEG) -> np.ndarray:
    """Baseline vectors (i < j) in the equatorial X, Y, Z frame, metres [n_bl, 3]."""
    lat = math.radians(lat_deg)
    n = enu.shape[0]
    ii, jj = np.triu_indices(n, k=1)
    d = enu[jj] - enu[ii]
    e, nn, u = d[:, 0], d[:, 1], d[:, 2]
    x = -math.sin(lat) * nn + math.cos(lat) * u
    y = e
    z = math.cos(lat) * nn + math.sin(lat) * u
    return np.stack([x, y, z], axis=1)


def hour_angles(n_int: int, span_h: float = 6.0) -> np.ndarray:
    """Integration centres in radians of hour angle over [-span/2, +span/2]."""
    t = (np.arange(n_int, dtype=np.float64) + 0.5) / n_int
    return (t - 0.5) * span_h * (2.0 * math.pi / 24.0)


def uvw_tracks(bxyz: np.ndarray, ha: np.ndarray, dec_deg: float = DEC_DEG) -> np.ndarray:
    """uvw in metres, rows time-major: [n_int * n_bl, 3]."""
    dec = math.radians(dec_deg)
    sh, ch = np.sin(ha)[:, None], np.cos(ha)[:, None]
    x, y, z = bxyz[None, :, 0], bxyz[None, :, 1], bxyz[None, :, 2]
    u = sh * x + ch * y
    v = -math.sin(dec) * ch * x + math.sin(dec) * sh * y + math.cos(dec) * z
    w = math.cos(dec) * ch * x - math.cos(dec) * sh * y + math.sin(dec) * z
    return np.stack([u, v, w], axis=-1).reshape(-1, 3)


def parallactic_angle(ha: np.ndarray, dec_deg: float = DEC_DEG, lat_deg: float = LAT_DEG) -> np.ndarray:
    dec, lat = math.radians(dec_deg), math.radians(lat_deg)
    return np.arctan2(np.sin(ha) * math.cos(lat),
                      math.sin(lat) * math.cos(dec) - math.cos(lat) * math.sin(dec) * np.cos(ha))


def channel_freqs(n_chan: int, f_lo: float = 2.0e9, f_hi: float = 4.0e9) -> np.ndarray:
    if n_chan == 1:
        return np.array([0.5 * (f_lo + f_hi)], dtype=np.float64)
    df = (f_hi - f_lo) / n_chan
    return f_lo + (np.arange(n_chan, dtype=np.float64) + 0.5) * df


def point_sources(n: int, radius_rad: float, seed: int = SEED_SKY, disk: bool = True):
    """n point sources, flux U(0.1, 1) Jy, uniform in a disk (or square) of the given radius."""
    rng = np.random.default_rng(seed)
    flux = rng.uniform(0.1, 1.0, n)
    if disk:
        r = radius_rad * np.sqrt(rng.uniform(0.0, 1.0, n))
        phi = rng.uniform(0.0, 2.0 * math.pi, n)
        l, m = r * np.cos(phi), r * np.sin(phi)
    else:
        l = rng.uniform(-radius_rad, radius_rad, n)
        m = rng.uniform(-radius_rad, radius_rad, n)
    return l.astype(np.float64), m.astype(np.float64), flux.astype(np.float64)


def point_source_vis(uvw_m, freq_hz, l, m, flux, device: Optional[str] = None, chunk_rows: int = 4096):
    """Exact visibilities of a point-source sky, complex128 [R, C] (numpy) or complex64 (torch device).

    V(u, v, w) = sum_k S_k exp(-2 pi i (u l_k + v m_k + w (n_k - 1))), u, v, w in wavelengths.
    The phase is formed in FP64 turns and reduced mod 1 before the exponential.
    """
    n_minus_1 = np.sqrt(1.0 - l * l - m * m) - 1.0
    if device is None or device == "cpu":
        R, C = uvw_m.shape[0], freq_hz.shape[0]
        out = np.zeros((R, C), dtype=np.complex128)
        for r0 in range(0, R, chunk_rows):
            r1 = min(R, r0 + chunk_rows)
            uvw = uvw_m[r0:r1]
            ph_m = (uvw[:, 0:1] * l[None, :] + uvw[:, 1:2] * m[None, :]
                    + uvw[:, 2:3] * n_minus_1[None, :])            # metres·(direction cosine)
            for c in range(C):
                t = ph_m * (freq_hz[c] / C_LIGHT)
                t = t - np.round(t)
                out[r0:r1, c] = (flux[None, :] * np.exp(-2j * math.pi * t)).sum(axis=1)
        return out
    import torch
    dev = torch.device(device)
    R, C = uvw_m.shape[0], freq_hz.shape[0]
    out = torch.zeros((R, C), dtype=torch.complex64, device=dev)
    L = torch.as_tensor(l, device=dev)
    M = torch.as_tensor(m, device=dev)
    NM = torch.as_tensor(n_minus_1, device=dev)
    S = torch.as_tensor(flux, device=dev, dtype=torch.float32)
    F = torch.as_tensor(freq_hz / C_LIGHT, device=dev)
    U = torch.as_tensor(uvw_m, device=dev)
    rows = max(1, (1 << 24) // max(1, C * L.numel()))
    for r0 in range(0, R, rows):
        r1 = min(R, r0 + rows)
        uvw = U[r0:r1]
        ph_m = uvw[:, 0:1] * L[None, :] + uvw[:, 1:2] * M[None, :] + uvw[:, 2:3] * NM[None, :]
        t = ph_m[:, None, :] * F[None, :, None]                      # [r, C, K] FP64 turns
        t = (t - torch.round(t)).to(torch.float32) * (2.0 * math.pi)
        out[r0:r1] = torch.complex((S * torch.cos(t)).sum(-1), (-S * torch.sin(t)).sum(-1))
    return out


@dataclasses.dataclass
class Workload:
    """One synthetic imaging workload; array layouts are those the C ABI takes."""
    name: str
    uvw_m: np.ndarray          # float64 [R, 3]
    freq_hz: np.ndarray        # float64 [C]
    pa_rad: np.ndarray         # float64 [R]
    n_bl: int
    n_int: int
    n_pol: int
    grid_n: int
    cell_rad: float
    du_lambda: float
    w_max_lambda: float
    oversampling: int
    ps_support: int
    use_w: bool
    n_wplanes: int
    use_a: bool
    n_pa_bins: int
    pa_bin_centers: np.ndarray  # float64 [n_pa]
    pa_bin: np.ndarray          # int32 [R]
    n_subbands: int
    subband_freq_hz: np.ndarray  # float64 [n_sb]
    chan_subband: np.ndarray     # int32 [C]
    max_support: int
    sky_l: np.ndarray
    sky_m: np.ndarray
    sky_flux: np.ndarray
    noise_sigma: float
    vis: object = None          # complex64 [R, C, P] (numpy or torch)
    weight: object = None       # float32 [R, C, P]

    @property
    def n_rows(self) -> int:
        return self.uvw_m.shape[0]

    @property
    def n_chan(self) -> int:
        return self.freq_hz.shape[0]

    @property
    def n_samples(self) -> int:
        return self.n_rows * self.n_chan


# Named configurations: the paper's VLA A-array S-band shape at several sizes.
CONFIGS = {
    # plain gridding, tiny: 351 baselines x 100 integrations, 1 channel at 3 GHz, 1 pol
    "standard": dict(n_int=100, n_chan=1, f_lo=2.5e9, f_hi=3.5e9, n_pol=1, grid_n=512, n_src=10,
                     src_radius_rad=math.radians(1.0 / 60.0), src_frac_fov=None, noise=0.0,
                     use_w=False, n_wplanes=1, use_a=False, n_pa=1, n_sb=1, max_support=7,
                     oversampling=20, ps_support=7),
    # W-projection: 351 x 2000 x 64 channels x 4 pols, 64 w-planes, supports 8-64, 4096^2 grid
    "wproj": dict(n_int=2000, n_chan=64, f_lo=2.0e9, f_hi=4.0e9, n_pol=4, grid_n=4096, n_src=200,
                  src_radius_rad=None, src_frac_fov=0.8, noise=1e-3, use_w=True, n_wplanes=64,
                  use_a=False, n_pa=1, n_sb=1, max_support=64, oversampling=20, ps_support=7),
    # batched AW-projection: same data, 20 PA bins x 32 w-planes x 16 sub-bands
    "awproj": dict(n_int=2000, n_chan=64, f_lo=2.0e9, f_hi=4.0e9, n_pol=4, grid_n=4096, n_src=200,
                   src_radius_rad=None, src_frac_fov=0.8, noise=1e-3, use_w=True, n_wplanes=32,
                   use_a=True, n_pa=20, n_sb=16, max_support=64, oversampling=20, ps_support=7),
    # differentiable forward model: 351 x 223 x 64 channels, 1 pol, supports 8-32, 1024^2 grid
    "autograd": dict(n_int=223, n_chan=64, f_lo=2.0e9, f_hi=4.0e9, n_pol=1, grid_n=1024, n_src=200,
                     src_radius_rad=None, src_frac_fov=0.8, noise=1e-3, use_w=True, n_wplanes=32,
                     use_a=False, n_pa=1, n_sb=1, max_support=32, oversampling=20, ps_support=7),
}


def make_workload(config: str, vis_device: Optional[str] = None, with_vis: bool = True, **overrides) -> Workload:
    """Build a named workload; keyword overrides shrink it (n_int, n_chan, grid_n, n_src, ...).

    Visibilities are computed on `vis_device` ("cpu"/None -> numpy complex64, "cuda" -> torch).
    """
    p = dict(CONFIGS[config])
    p.update(overrides)
    enu = antenna_enu()
    bxyz = baselines_xyz(enu)
    n_bl = bxyz.shape[0]
    ha = hour_angles(p["n_int"])
    uvw = uvw_tracks(bxyz, ha)
    pa_t = parallactic_angle(ha)
    pa = np.repeat(pa_t, n_bl)
    freq = channel_freqs(p["n_chan"], p["f_lo"], p["f_hi"])
    lam_min = C_LIGHT / freq.max()
    u_max = float(np.max(np.abs(uvw[:, :2]))) / lam_min
    w_max = float(np.max(np.abs(uvw[:, 2]))) / lam_min
    N = int(p["grid_n"])
    du = 2.0 * u_max / (N - p["max_support"] - 4)
    cell = 1.0 / (N * du)

    n_pa = int(p["n_pa"])
    if n_pa > 1:
        lo, hi = float(pa_t.min()), float(pa_t.max())
        edges = np.linspace(lo, hi, n_pa + 1)
        centers = 0.5 * (edges[:-1] + edges[1:])
        bins_t = np.clip(np.searchsorted(edges, pa_t, side="right") - 1, 0, n_pa - 1)
    else:
        centers = np.array([float(np.median(pa_t))])
        bins_t = np.zeros(p["n_int"], dtype=np.int64)
    pa_bin = np.repeat(bins_t, n_bl).astype(np.int32)

    n_sb = int(p["n_sb"])
    C = freq.shape[0]
    chan_sb = (np.arange(C) * n_sb // C).astype(np.int32) if n_sb > 1 else np.zeros(C, dtype=np.int32)
    sb_freq = np.array([freq[chan_sb == s].mean() for s in range(n_sb)], dtype=np.float64)

    fov_half = 0.5 * N * cell
    radius = p["src_radius_rad"] if p["src_radius_rad"] is not None else p["src_frac_fov"] * fov_half
    l, m, flux = point_sources(int(p["n_src"]), radius, disk=p["src_radius_rad"] is not None)

    wl = Workload(
        name=config, uvw_m=uvw, freq_hz=freq, pa_rad=pa, n_bl=n_bl, n_int=int(p["n_int"]),
        n_pol=int(p["n_pol"]), grid_n=N, cell_rad=cell, du_lambda=du, w_max_lambda=w_max,
        oversampling=int(p["oversampling"]), ps_support=int(p["ps_support"]), use_w=bool(p["use_w"]),
        n_wplanes=int(p["n_wplanes"]), use_a=bool(p["use_a"]), n_pa_bins=n_pa, pa_bin_centers=centers,
        pa_bin=pa_bin, n_subbands=n_sb, subband_freq_hz=sb_freq, chan_subband=chan_sb,
        max_support=int(p["max_support"]), sky_l=l, sky_m=m, sky_flux=flux, noise_sigma=float(p["noise"]))
    if with_vis:
        fill_visibilities(wl, device=vis_device)
    return wl


def fill_visibilities(wl: Workload, device: Optional[str] = None) -> None:
    """Sky + noise visibilities and natural weights for all pols (see module docstring)."""
    R, C, P = wl.n_rows, wl.n_chan, wl.n_pol
    rng = np.random.default_rng(SEED_NOISE)
    sig_bl = rng.uniform(0.8, 1.2, wl.n_bl) * (wl.noise_sigma if wl.noise_sigma > 0 else 1e-3)
    sig_row = np.tile(sig_bl, wl.n_int)                    # rows are time-major
    w_row = (1.0 / (sig_row * sig_row)).astype(np.float32)
    sky = point_source_vis(wl.uvw_m, wl.freq_hz, wl.sky_l, wl.sky_m, wl.sky_flux, device=device)
    sky_pol = [0, 3] if P == 4 else ([0, 1] if P == 2 else [0])
    if device is None or device == "cpu":
        vis = np.zeros((R, C, P), dtype=np.complex64)
        for p in sky_pol:
            vis[:, :, p] = sky
        if wl.noise_sigma > 0:
            for p in range(P):
                nr = rng.standard_normal((R, C)).astype(np.float32)
                ni = rng.standard_normal((R, C)).astype(np.float32)
                vis[:, :, p] += (nr + 1j * ni).astype(np.complex64) * sig_row[:, None].astype(np.float32)
        weight = np.broadcast_to(w_row[:, None, None], (R, C, P)).astype(np.float32).copy()
        wl.vis, wl.weight = vis, weight
        return
    import torch
    dev = torch.device(device)
    g = torch.Generator(device=dev)
    g.manual_seed(SEED_NOISE)
    vis = torch.zeros((R, C, P), dtype=torch.complex64, device=dev)
    for p in sky_pol:
        vis[:, :, p] = sky
    sig = torch.as_tensor(sig_row, device=dev, dtype=torch.float32)
    if wl.noise_sigma > 0:
        for p in range(P):
            nr = torch.randn((R, C), generator=g, device=dev, dtype=torch.float32)
            ni = torch.randn((R, C), generator=g, device=dev, dtype=torch.float32)
            vis[:, :, p] += torch.complex(nr, ni) * sig[:, None]
    w = torch.as_tensor(w_row, device=dev)
    wl.vis = vis
    wl.weight = w[:, None, None].expand(R, C, P).contiguous()


def gaussian_blob_sky(n: int, cell_rad: float, l, m, flux, seed: int = SEED_SKY) -> np.ndarray:
    """Float32 [n, n] sky image: rasterised point sources plus one Gaussian blob (autograd workload)."""
    img = np.zeros((n, n), dtype=np.float64)
    ix = np.clip(np.round(l / cell_rad).astype(np.int64) + n // 2, 0, n - 1)
    iy = np.clip(np.round(m / cell_rad).astype(np.int64) + n // 2, 0, n - 1)
    np.add.at(img, (iy, ix), flux)
    rng = np.random.default_rng(seed + 100)
    cx, cy = rng.uniform(-0.2, 0.2, 2) * n
    yy, xx = np.mgrid[0:n, 0:n] - n // 2
    img += 0.5 * np.exp(-((xx - cx) ** 2 + (yy - cy) ** 2) / (2.0 * (0.02 * n) ** 2))
    return img.astype(np.float32)


def baseline_antennas(n_ant: int = 27):
    """Antenna indices (ant1 < ant2) of the baselines in the order baselines_xyz produces them."""
    a1, a2 = np.triu_indices(n_ant, k=1)
    return a1.astype(np.int32), a2.astype(np.int32)


def antenna_gains(shape, seed: int = 5) -> np.ndarray:
    """Seeded complex antenna gains: amplitude U(0.8, 1.2), phase U(-pi, pi); complex128 [shape]."""
    rng = np.random.default_rng(seed)
    return rng.uniform(0.8, 1.2, shape) * np.exp(1j * rng.uniform(-np.pi, np.pi, shape))
