"""The synthetic inputs follow their stated recipe (host only): the VLA-like Y layout and its 351
baselines, uvw tracks that are rotations of the baselines, the hour-angle span, the 2-4 GHz channel
grid and its sub-bands, the parallactic-angle bins, natural weights from the per-baseline noise,
the source fields, and the full sizes of the W-projection and batched AW-projection workloads.
They stand in for the paper's VLA A-array S-band data (Sec. 6), which is not available."""
import math

import numpy as np
import pytest

import synth


def test_layout_is_a_y_of_27_antennas():
    enu = synth.antenna_enu()
    assert enu.shape == (27, 3) and np.all(enu[:, 2] == 0.0)
    r = np.hypot(enu[:, 0], enu[:, 1])
    az = np.degrees(np.arctan2(enu[:, 0], enu[:, 1])) % 360.0
    for arm, angle in enumerate((5.0, 125.0, 245.0)):
        sl = slice(9 * arm, 9 * arm + 9)
        assert np.allclose(az[sl], angle, atol=1e-9)
        nominal = 21000.0 * (np.arange(1, 10) / 9.0) ** 1.716
        assert np.all(np.abs(r[sl] / nominal - 1.0) <= 0.005 + 1e-12)
    assert np.array_equal(enu, synth.antenna_enu())          # seeded


def test_uvw_tracks_rotate_the_baselines():
    bxyz = synth.baselines_xyz(synth.antenna_enu())
    assert bxyz.shape == (351, 3)
    ha = synth.hour_angles(2000)
    assert ha.shape == (2000,)
    assert ha[0] == pytest.approx(-3.0 * math.pi / 12.0 * (1.0 - 1.0 / 2000.0))
    assert np.allclose(ha + ha[::-1], 0.0, atol=1e-15)       # symmetric about transit
    uvw = synth.uvw_tracks(bxyz, ha[::100])
    assert uvw.shape == (20 * 351, 3)
    # an orthogonal rotation of each baseline: lengths are kept; rows are time-major
    lb = np.linalg.norm(bxyz, axis=1)
    assert np.allclose(np.linalg.norm(uvw, axis=1).reshape(20, 351), lb[None, :], rtol=1e-12)
    assert np.all(lb <= 2 * 21000.0 * 1.005)


def test_channels_subbands_and_pa_bins():
    wl = synth.make_workload("awproj", with_vis=False, n_int=40)
    assert np.allclose(wl.freq_hz, 2.0e9 + (np.arange(64) + 0.5) * 31.25e6, rtol=0, atol=1e-3)
    assert np.array_equal(wl.chan_subband, np.arange(64) // 4)
    assert np.allclose(wl.subband_freq_hz, wl.freq_hz.reshape(16, 4).mean(axis=1))
    assert wl.n_pa_bins == 20 and np.all(np.diff(wl.pa_bin_centers) > 0)
    assert wl.pa_bin.min() >= 0 and wl.pa_bin.max() == 19
    # rows are time-major: every baseline of one integration shares its bin
    assert np.all(wl.pa_bin.reshape(40, 351) == wl.pa_bin.reshape(40, 351)[:, :1])


def test_full_workload_sizes():
    for name in ("wproj", "awproj"):
        wl = synth.make_workload(name, with_vis=False)
        assert (wl.n_rows, wl.n_chan, wl.n_pol, wl.grid_n) == (702000, 64, 4, 4096)
        assert wl.n_rows * wl.n_chan * wl.n_pol == 179712000
        assert wl.max_support == 64 and wl.oversampling == 20
    assert synth.make_workload("wproj", with_vis=False).n_wplanes == 64
    aw = synth.make_workload("awproj", with_vis=False)
    assert (aw.n_pa_bins, aw.n_wplanes, aw.n_subbands) == (20, 32, 16)
    ag = synth.make_workload("autograd", with_vis=False)
    assert (ag.n_rows * ag.n_chan, ag.n_pol, ag.grid_n) == (5009472, 1, 1024)


def test_sky_noise_and_natural_weights():
    wl = synth.make_workload("wproj", n_int=20, n_chan=4, grid_n=512, n_wplanes=4, max_support=32)
    assert wl.sky_flux.shape == (200,) and wl.sky_flux.min() >= 0.1 and wl.sky_flux.max() <= 1.0
    assert np.hypot(wl.sky_l, wl.sky_m).max() <= 0.8 * 0.5 * wl.grid_n * wl.cell_rad * math.sqrt(2) + 1e-15
    # per-baseline sigma in [0.8, 1.2] mJy; weight = 1 / sigma^2 for every pol
    w = wl.weight.reshape(wl.n_int, wl.n_bl, wl.n_chan, 4)
    assert np.all(w == w[:1, :, :1, :1])
    sigma = 1.0 / np.sqrt(w[0, :, 0, 0].astype(np.float64))
    assert sigma.min() >= 0.8e-3 * (1 - 1e-6) and sigma.max() <= 1.2e-3 * (1 + 1e-6)
    # RL and LR carry noise only: real and imaginary parts of V / sigma have unit variance
    v = wl.vis.reshape(wl.n_int, wl.n_bl, wl.n_chan, 4)[..., 1:3] / sigma[None, :, None, None]
    for part in (v.real, v.imag):
        assert abs(float(part.std()) - 1.0) < 0.02 and abs(float(part.mean())) < 0.02
    # RR and LL carry the sky (the same in both) plus independent noise
    d = wl.vis[..., 0] - wl.vis[..., 3]
    assert abs(float(np.std(d.real / np.repeat(np.tile(sigma, wl.n_int), 1)[:, None])) - math.sqrt(2)) < 0.05


def test_point_source_visibilities():
    l, m, f = np.array([1e-3, -2e-3]), np.array([5e-4, 1e-3]), np.array([0.5, 0.25])
    uvw = np.array([[0.0, 0.0, 0.0], [120.0, -80.0, 15.0], [-120.0, 80.0, -15.0]])
    freq = np.array([synth.C_LIGHT])                           # u in wavelengths = u in metres
    v = synth.point_source_vis(uvw, freq, l, m, f)[:, 0]
    assert v[0] == pytest.approx(0.75)                         # zero spacing: total flux
    assert v[2] == pytest.approx(np.conj(v[1]))                # V(-u) = conj V(u) for a real sky
    n1 = np.sqrt(1 - l * l - m * m) - 1
    ref = (f * np.exp(-2j * math.pi * (120.0 * l - 80.0 * m + 15.0 * n1))).sum()
    assert v[1] == pytest.approx(ref, rel=1e-12)
