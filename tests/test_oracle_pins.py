"""Pins of the FP64 oracle against what the paper and mathematics fix (CPU only).

Each test checks the oracle against something other than itself: an integral
equation, a library routine, a closed form, an exact identity, brute force, or a
convergence law.  They are chosen so that a dropped term, a wrong sign, a wrong index
or a transposed operand anywhere in ``oracle/`` fails at least one of them.
"""
import math

import numpy as np
import pytest
from scipy.special import pro_ang1, pro_cv

import synth
from oracle import cf, image, index, ops, pswf


# ---------------------------------------------------------------- PSWF (Tab. AWP-CFSETUP PS term)

@pytest.mark.parametrize("W", [4, 5, 6, 7, 8])
def test_pswf_integral_equation(W):
    """psi_0 is an eigenfunction of the finite Fourier transform on [-1, 1]."""
    c = pswf.pswf_c(W)
    t, wq = np.polynomial.legendre.leggauss(200)
    pt = pswf.psi0(c, t)
    x = np.linspace(-1.0, 1.0, 17)
    ratio = np.array([(wq * np.exp(1j * c * xx * t) * pt).sum() / pswf.psi0(c, xx) for xx in x])
    assert np.all(np.abs(ratio.imag) < 1e-10)
    assert np.ptp(ratio.real) / abs(ratio.real.mean()) < 1e-10
    # energy concentration lambda_0 = c |mu|^2 / (2 pi) of the ground state is just below 1
    lam = c * abs(ratio.real.mean()) ** 2 / (2 * math.pi)
    assert 0.99 < lam < 1.0


@pytest.mark.parametrize("W", [5, 7, 8])
def test_pswf_matches_library(W):
    """Characteristic value and shape agree with scipy's pro_cv / pro_ang1."""
    c = pswf.pswf_c(W)
    chi, _ = pswf.legendre_coeffs(c)
    assert abs(chi - pro_cv(0, 0, c)) < 1e-9 * max(1.0, abs(chi))
    x = np.linspace(0.0, 0.9, 10)
    ref = pro_ang1(0, 0, c, x)[0] / pro_ang1(0, 0, c, 0.0)[0]
    assert np.allclose(pswf.taper(W, x), ref, rtol=1e-9, atol=1e-12)


def test_pswf_ground_state_has_no_zero():
    c = pswf.pswf_c(7)
    x = np.linspace(-1, 1, 2001)
    assert np.all(pswf.psi0(c, x) > 0)
    assert pswf.taper(7, 0.0) == pytest.approx(1.0, abs=1e-15)


# ---------------------------------------------------------------- CFs

def _params(**kw):
    base = dict(grid_n=256, cell_rad=2e-6, oversampling=8, ps_support=7, max_support=16)
    base.update(kw)
    return cf.CFParams(**base)


def test_cf_ps_matches_closed_form():
    """PS-only CF equals the continuous transform of the taper: (mu/2) psi_0(2 du / W) / psi_0(0)."""
    W = 7
    p = _params(max_support=8, oversampling=4, ps_support=W)
    tab = cf.cf_table(p, 0, 0, 0)
    c = pswf.pswf_c(W)
    t, wq = np.polynomial.legendre.leggauss(200)
    mu = (wq * pswf.psi0(c, t)).sum() / pswf.psi0(c, 0.0)      # integral at x = 0, normalised
    du = cf.tap_positions(8, 4)                                # [o, t]
    for oy in range(5):
        for ox in range(5):
            ref_u = 0.5 * mu * pswf.psi0(c, np.clip(2 * du[ox] / W, -1, 1)) / pswf.psi0(c, 0.0)
            ref_v = 0.5 * mu * pswf.psi0(c, np.clip(2 * du[oy] / W, -1, 1)) / pswf.psi0(c, 0.0)
            inside = (np.abs(du[oy])[:, None] <= W / 2) & (np.abs(du[ox])[None, :] <= W / 2)
            ref = ref_v[:, None] * ref_u[None, :]
            err = np.abs(tab[oy, ox] - ref)[inside]
            assert err.max() < 2e-3 * ref.max()
            # the screen grid holds x = -N/2 but not +N/2: that one edge sample gives the
            # only imaginary part, at most T(edge) / M per axis
            assert np.abs(tab[oy, ox].imag).max() < 2 * pswf.taper(W, 1.0) / cf.screen_size(8)


@pytest.mark.parametrize("mode", ["ps", "ps_w", "ps_a", "ps_a_w"])
def test_cf_inverts_to_screen(mode):
    """The S taps of every offset transform back to the image-plane product of the terms.

    sum_t c(du_t, dv_t) exp(+2 pi i (du x + dv y) / N) = screen(x, y) at the screen points,
    which fixes the transform sign, the tap positions, the axis order and each term.
    """
    use_w = "w" in mode
    use_a = "a" in mode
    # a 0.3 deg field: the W phase reaches ~0.1 turn and the A-term falls to ~0.3 at its edge
    p = _params(cell_rad=2e-5, use_w=use_w, n_wplanes=3, w_max_lambda=3.0e4, use_a=use_a, n_pa_bins=1,
                pa_bin_centers=[0.7], n_subbands=1, subband_freq_hz=[3.0e9], max_support=24,
                oversampling=4)
    ks = p.n_signed - 1 if use_w else 0          # the most positive w plane
    tab = cf.cf_table(p, 0, 0, ks)
    S = tab.shape[-1]
    M = cf.screen_size(S)
    scr = cf.screen(p, 0, 0, ks, M)
    du = cf.tap_positions(S, p.oversampling)
    pts = [(M // 2, M // 2), (M // 2 + 3, M // 2 - 25), (M // 2 - 27, M // 2 + 2), (M // 2 + 26, M // 2 + 19)]
    for (iy, ix) in pts:
        x = (ix - M / 2) * p.grid_n / M
        y = (iy - M / 2) * p.grid_n / M
        for oy, ox in [(0, 0), (1, 3), (4, 2)]:
            eu = np.exp(2j * math.pi * du[ox] * x / p.grid_n)
            ev = np.exp(2j * math.pi * du[oy] * y / p.grid_n)
            back = ev @ tab[oy, ox] @ eu
            # the edge sample of the screen (T ~ 3e-4 there) leaks outside the S taps
            assert abs(back - scr[iy, ix]) < 2e-5


def test_cf_negative_w_is_conjugate_reflection():
    """screen(-w) = conj(screen(w)) and T, A are real, so c_{-w}(d) = conj(c_w(-d)):
    table_{-w}[oy, ox, ty, tx] = conj(table_w[OS-oy, OS-ox, S-1-ty, S-1-tx])."""
    p = _params(use_w=True, n_wplanes=4, w_max_lambda=5e4, use_a=True, pa_bin_centers=[0.3],
                subband_freq_hz=[2.5e9], max_support=32, oversampling=6)
    for k in (1, 3):
        tp = cf.cf_table(p, 0, 0, p.n_wplanes - 1 + k)
        tn = cf.cf_table(p, 0, 0, p.n_wplanes - 1 - k)
        ref = np.conj(tp[::-1, ::-1, ::-1, ::-1])
        assert np.abs(tn - ref).max() < 1e-13 * np.abs(tp).max()


def test_cf_unit_sum_and_support_schedule():
    p = _params(max_support=8, oversampling=20)
    tab = cf.cf_table(p, 0, 0, 0)
    # even S: offset 0 puts the taps on integer distances; the kernel sums to T(0) = 1
    assert abs(tab[0, 0].sum() - 1.0) < 1e-3
    pw = _params(use_w=True, n_wplanes=64, w_max_lambda=1e5, max_support=64)
    s = [cf.support_of_plane(pw, pw.n_wplanes - 1 + k) for k in range(64)]
    assert s[0] == 8 and s[-1] == 64 and all(a <= b for a, b in zip(s, s[1:]))
    assert all(v % 8 == 0 for v in s)
    assert cf.support_of_plane(pw, 0) == 64      # the most negative plane mirrors the most positive


# ---------------------------------------------------------------- index rules

def test_index_tap_distance_matches_cf_positions():
    """Tap t of a kept sample sits at sample-minus-pixel distance within 1/(2 OS) of du[ox, t]."""
    wl = synth.make_workload("standard", n_int=6, with_vis=False)
    for S, OS in [(7, 20), (8, 20), (1, 1), (24, 7)]:
        p = cf.CFParams(grid_n=wl.grid_n, cell_rad=wl.cell_rad, oversampling=OS, max_support=S, ps_support=min(S, 7))
        idx = index.sample_index(p, wl.uvw_m, wl.freq_hz)
        sc = wl.freq_hz / synth.C_LIGHT
        x = (wl.uvw_m[:, 0:1] * sc * (wl.grid_n * wl.cell_rad) + wl.grid_n // 2).reshape(-1)
        v = idx.valid
        assert v.mean() > 0.95
        du = cf.tap_positions(S, OS)
        for t in (0, S // 2, S - 1):
            dist = x[v] - (idx.p0x[v] + t)
            assert np.all(np.abs(dist - du[idx.ox[v], t]) <= 0.5 / OS + 1e-9)
        assert idx.ox.min() >= 0 and idx.ox.max() <= OS
        assert np.all(idx.p0x[v] >= 0) and np.all(idx.p0x[v] + S <= wl.grid_n)


def test_index_wplane_and_drop_rules():
    wl = synth.make_workload("wproj", n_int=8, n_chan=4, grid_n=1024, with_vis=False)
    p = cf.CFParams(grid_n=wl.grid_n, cell_rad=wl.cell_rad, use_w=True, n_wplanes=16,
                    w_max_lambda=wl.w_max_lambda, max_support=32)
    idx = index.sample_index(p, wl.uvw_m, wl.freq_hz)
    w = (wl.uvw_m[:, 2:3] * wl.freq_hz[None, :] / synth.C_LIGHT).reshape(-1)
    ks = idx.cf - (p.n_wplanes - 1)
    wk = ks * p.w_max_lambda / (p.n_wplanes - 1)
    dw = p.w_max_lambda / (p.n_wplanes - 1)
    v = idx.valid
    assert np.all(np.abs(w[v] - wk[v]) <= 0.5 * dw * (1 + 1e-12))
    assert np.all(np.sign(ks[v & (np.abs(w) > dw)]) == np.sign(w[v & (np.abs(w) > dw)]))
    # a sample pushed off the grid is dropped; one pushed beyond w_max is dropped
    uvw = wl.uvw_m[:4].copy()
    uvw[0, 0] = 1e9
    uvw[1, 2] = 10 * wl.w_max_lambda * synth.C_LIGHT / wl.freq_hz.max()
    idx2 = index.sample_index(p, uvw, wl.freq_hz[:1])
    assert not idx2.valid[0] and not idx2.valid[1]


# ---------------------------------------------------------------- G and D

def _random_index(n, N, S, OS, n_cf, rng):
    p0 = rng.integers(0, N - S + 1, size=(2, n))
    return index.SampleIndex(valid=rng.random(n) > 0.1, cf=rng.integers(0, n_cf, n).astype(np.int32),
                             p0x=p0[0], p0y=p0[1], ox=rng.integers(0, OS + 1, n).astype(np.int32),
                             oy=rng.integers(0, OS + 1, n).astype(np.int32),
                             support=np.full(n, S, dtype=np.int32))


def test_delta_cf_is_direct_binning(oracle_built):
    """Support-1 CF equal to 1: G is nearest-pixel binning, D is direct lookup (exact)."""
    wl = synth.make_workload("standard", n_int=20, with_vis=True)
    N = wl.grid_n
    p = cf.CFParams(grid_n=N, cell_rad=wl.cell_rad, oversampling=1, ps_support=1, use_ps=False, max_support=1)
    idx = index.sample_index(p, wl.uvw_m, wl.freq_hz)
    buf = np.ones(4, dtype=np.complex128)           # (OS+1)^2 offsets x 1 tap
    off = np.zeros(1, dtype=np.int64)
    vis = wl.vis.reshape(-1, 1).astype(np.complex128)
    wt = wl.weight.reshape(-1, 1).astype(np.float64)
    g, sw = ops.grid(idx, buf, off, 1, N, vis, wt)
    sc = wl.freq_hz / synth.C_LIGHT
    u = (wl.uvw_m[:, 0:1] * sc).reshape(-1)
    v = (wl.uvw_m[:, 1:2] * sc).reshape(-1)
    ix = np.floor(u / wl.du_lambda + N // 2 + 0.5).astype(np.int64)
    iy = np.floor(v / wl.du_lambda + N // 2 + 0.5).astype(np.int64)
    ref = np.zeros((N, N), dtype=np.complex128)
    np.add.at(ref, (iy, ix), wt[:, 0] * vis[:, 0])
    assert np.array_equal(g[:, :, 0], ref)
    assert sw[0] == wt.sum()
    rng = np.random.default_rng(7)
    X = rng.standard_normal((N, N, 1)) + 1j * rng.standard_normal((N, N, 1))
    d = ops.degrid(idx, buf, off, 1, X)
    assert np.array_equal(d[:, 0], X[iy, ix, 0])


@pytest.mark.parametrize("P", [1, 4])
def test_adjoint_dot_product(oracle_built, P):
    """<G V, X> = <V, D X> for random complex V, X, random (non-symmetric) CF tables."""
    rng = np.random.default_rng(11 + P)
    N, S, OS, n_cf, n = 48, 9, 3, 3, 400
    idx = _random_index(n, N, S, OS, n_cf, rng)
    per = (OS + 1) ** 2 * S * S
    buf = rng.standard_normal(per * n_cf) + 1j * rng.standard_normal(per * n_cf)
    off = np.arange(n_cf, dtype=np.int64) * per
    idx.phasor = np.exp(2j * math.pi * rng.random(n))
    V = rng.standard_normal((n, P)) + 1j * rng.standard_normal((n, P))
    X = rng.standard_normal((N, N, P)) + 1j * rng.standard_normal((N, N, P))
    gv, _ = ops.grid(idx, buf, off, OS, N, V, np.ones((n, P)))
    dx = ops.degrid(idx, buf, off, OS, X)
    a, b = np.vdot(gv, X), np.vdot(V, dx)
    assert abs(a - b) <= 1e-12 * abs(a)
    # the numpy restatement agrees with the C loops
    gv2, _ = ops.grid_numpy(idx, buf, off, OS, N, V, np.ones((n, P)))
    assert np.abs(gv - gv2).max() < 1e-12 * np.abs(gv).max()
    assert np.abs(dx - ops.degrid_numpy(idx, buf, off, OS, X)).max() < 1e-12 * np.abs(dx).max()


def test_linearity_and_partition(oracle_built):
    """G(aV1 + bV2) = a G(V1) + b G(V2); the sum over sample partitions equals the whole."""
    rng = np.random.default_rng(21)
    N, S, OS, n_cf, n, P = 40, 8, 4, 2, 300, 2
    idx = _random_index(n, N, S, OS, n_cf, rng)
    per = (OS + 1) ** 2 * S * S
    buf = rng.standard_normal(per * n_cf) + 1j * rng.standard_normal(per * n_cf)
    off = np.arange(n_cf, dtype=np.int64) * per
    V1 = rng.standard_normal((n, P)) + 1j * rng.standard_normal((n, P))
    V2 = rng.standard_normal((n, P)) + 1j * rng.standard_normal((n, P))
    w = rng.random((n, P))
    a, b = 0.7 - 0.2j, -1.3 + 0.5j
    g1, _ = ops.grid(idx, buf, off, OS, N, V1, w)
    g2, _ = ops.grid(idx, buf, off, OS, N, V2, w)
    g12, _ = ops.grid(idx, buf, off, OS, N, a * V1 + b * V2, w)
    assert np.abs(g12 - (a * g1 + b * g2)).max() < 1e-12 * np.abs(g12).max()
    parts = np.array_split(np.arange(n), 3)
    tot = np.zeros_like(g1)
    sw_tot = np.zeros(P)
    for prt in parts:
        sub = index.SampleIndex(valid=idx.valid[prt], cf=idx.cf[prt], p0x=idx.p0x[prt], p0y=idx.p0y[prt],
                                ox=idx.ox[prt], oy=idx.oy[prt], support=idx.support[prt])
        gp, swp = ops.grid(sub, buf, off, OS, N, V1[prt], w[prt])
        tot += gp
        sw_tot += swp
    _, sw = ops.grid(idx, buf, off, OS, N, V1, w)
    assert np.abs(tot - g1).max() < 1e-12 * np.abs(g1).max()
    assert np.allclose(sw_tot, sw, rtol=1e-14)


def _standard_case(OS, n_int=30, w_scale=1.0, use_w=False, n_wplanes=1, seed=5):
    wl = synth.make_workload("standard", n_int=n_int, with_vis=False)
    uvw = wl.uvw_m.copy()
    uvw[:, 2] *= w_scale
    N = wl.grid_n
    rng = np.random.default_rng(seed)
    l = rng.uniform(-150, 150, 6) * wl.cell_rad if use_w else rng.uniform(-60, 60, 6) * wl.cell_rad
    m = rng.uniform(-150, 150, 6) * wl.cell_rad if use_w else rng.uniform(-60, 60, 6) * wl.cell_rad
    fl = rng.uniform(0.1, 1, 6)
    vis = image.point_source_vis(uvw, wl.freq_hz, l, m, fl)
    wmax = float(np.abs(uvw[:, 2]).max() * wl.freq_hz.max() / synth.C_LIGHT)
    p = cf.CFParams(grid_n=N, cell_rad=wl.cell_rad, oversampling=OS, ps_support=7,
                    use_w=use_w, n_wplanes=n_wplanes, w_max_lambda=wmax, max_support=(24 if use_w else 7))
    tabs = cf.cf_set(p)
    buf, off, _ = cf.flatten_cf_set(p, tabs)
    idx = index.sample_index(p, uvw, wl.freq_hz)
    assert idx.valid.mean() > 0.97
    # dropped samples (footprint off the grid) carry no weight in either image
    wt = idx.valid.reshape(vis.shape).astype(np.float64)
    g, sw = ops.grid(idx, buf, off, OS, N, vis.reshape(-1, 1), wt.reshape(-1, 1))
    img = image.dirty_image(g, sw, 7)[:, :, 0]
    sx = np.round(l / wl.cell_rad).astype(int) + N // 2
    sy = np.round(m / wl.cell_rad).astype(int) + N // 2
    gy, gx = np.meshgrid(np.arange(N // 2 - 64, N // 2 + 64, 8), np.arange(N // 2 - 64, N // 2 + 64, 8), indexing="ij")
    py = np.concatenate([sy, gy.ravel()])
    px = np.concatenate([sx, gx.ravel()])
    return wl, uvw, vis, wt, img, py, px


def test_fft_image_matches_dft_and_converges_with_oversampling(oracle_built):
    """G, F-dagger and the taper correction reproduce the brute-force 2-D DFT image; the error
    is set by the oversampling quantisation and shrinks as OS grows."""
    errs = {}
    for OS in (20, 400):
        wl, uvw, vis, wt, img, py, px = _standard_case(OS)
        dft = image.dft_dirty_image(uvw, wl.freq_hz, vis, wt, wl.grid_n, wl.cell_rad, py, px, with_w=False)
        errs[OS] = np.abs(img[py, px] - dft).max() / np.abs(dft).max()
    assert errs[20] < 1e-3
    assert errs[400] < errs[20] / 8


def test_wprojection_corrects_noncoplanar_baselines(oracle_built):
    """With the exact w-term in the data, W-projection matches the DFT image that includes
    w (n - 1); plain gridding of the same data does not."""
    out = {}
    for use_w in (False, True):
        wl, uvw, vis, wt, img, py, px = _standard_case(100, w_scale=8.0, use_w=use_w, n_wplanes=(16 if use_w else 1))
        dft = image.dft_dirty_image(uvw, wl.freq_hz, vis, wt, wl.grid_n, wl.cell_rad, py, px, with_w=True)
        out[use_w] = np.abs(img[py, px] - dft).max() / np.abs(dft).max()
    assert out[True] < 5e-3
    assert out[True] < out[False] / 5


def test_chi2_gradient_matches_central_differences(oracle_built):
    """Eq. ImChisq and Eq. ResIm: the gradient of chi^2(I) = sum w |V - D F T^-1 I|^2 over the real
    image I is -2 Re[T^-1 F^H G W (V - D F T^-1 I)], with G = D^H (unit weights) and F^H the
    unnormalised inverse transform.  chi^2 is quadratic in I, so a central difference with any step
    carries rounding only (FP64).  A missing N^2 in F^H, one taper division instead of two, or a
    flipped sign fails it."""
    wl = synth.make_workload("autograd", n_int=3, n_chan=2, grid_n=128, n_src=5, n_wplanes=4, max_support=16)
    N = wl.grid_n
    p = cf.CFParams(grid_n=N, cell_rad=wl.cell_rad, oversampling=wl.oversampling, ps_support=wl.ps_support,
                    use_w=True, n_wplanes=wl.n_wplanes, w_max_lambda=wl.w_max_lambda, max_support=wl.max_support)
    idx = index.sample_index(p, wl.uvw_m, wl.freq_hz)
    assert idx.valid.all()
    buf, off, _ = cf.flatten_cf_set(p, cf.cf_set(p, which=set(np.unique(idx.cf).tolist())))
    V = wl.vis.reshape(-1, 1).astype(np.complex128)
    w = wl.weight.reshape(-1, 1).astype(np.float64)
    inner = np.zeros((N, N, 1))
    inner[N // 4:3 * N // 4, N // 4:3 * N // 4] = 1.0
    rng = np.random.default_rng(synth.SEED_FD)
    I0 = rng.standard_normal((N, N, 1)) * inner

    def model_vis(I):
        return ops.degrid(idx, buf, off, p.oversampling, image.model_to_grid(I, p.ps_support))

    def chi2(I):
        r = V - model_vis(I)
        return float((w * (r.real ** 2 + r.imag ** 2)).sum())

    g, _ = ops.grid(idx, buf, off, p.oversampling, N, w * (V - model_vis(I0)), np.ones_like(w))
    t = image.taper_image(N, p.ps_support)
    grad = -2.0 * (image.grid_to_image(g) / (t[:, None] * t[None, :])[:, :, None]).real
    for _ in range(3):
        d = rng.standard_normal(I0.shape) * inner
        eps = float(np.linalg.norm(I0) / np.linalg.norm(d))
        fd = (chi2(I0 + eps * d) - chi2(I0 - eps * d)) / (2.0 * eps)
        an = float((grad * d).sum())
        assert abs(fd - an) <= 1e-8 * abs(an), (fd, an)


def test_degrid_model_matches_analytic_visibilities(oracle_built):
    """D of F(model / T T) for point sources at pixel centres ~ their analytic visibilities."""
    wl = synth.make_workload("standard", n_int=10, with_vis=False)
    N = wl.grid_n
    p = cf.CFParams(grid_n=N, cell_rad=wl.cell_rad, oversampling=100, ps_support=7, max_support=7)
    buf, off, _ = cf.flatten_cf_set(p, cf.cf_set(p))
    model = np.zeros((N, N, 1))
    pix = [(N // 2, N // 2, 1.0), (N // 2 + 20, N // 2 - 33, 0.5), (N // 2 - 41, N // 2 + 12, 0.25)]
    for (y, x, f) in pix:
        model[y, x, 0] = f
    gridc = image.model_to_grid(model, 7)
    idx = index.sample_index(p, wl.uvw_m, wl.freq_hz)
    d = ops.degrid(idx, buf, off, 100, gridc)[:, 0]
    l = np.array([(x - N // 2) * wl.cell_rad for (y, x, f) in pix])
    m = np.array([(y - N // 2) * wl.cell_rad for (y, x, f) in pix])
    fl = np.array([f for (_, _, f) in pix])
    uvw2 = wl.uvw_m.copy()
    uvw2[:, 2] = 0.0                                 # plain 2-D degridding has no w-term
    ref = image.point_source_vis(uvw2, wl.freq_hz, l, m, fl)[:, 0]
    assert np.abs(d - ref).max() < 2e-3 * fl.sum()


# ------------------------------------------------------------------------------------ Hogbom CLEAN

def _compact_psf(Np, half=4, width=4.0):
    yy, xx = np.mgrid[0:Np, 0:Np]
    psf = np.exp(-(((yy - Np // 2) ** 2 + (xx - Np // 2) ** 2) / width)).astype(np.float32)
    psf[np.abs(yy - Np // 2) > half] = 0
    psf[np.abs(xx - Np // 2) > half] = 0
    return psf


def _place(psf, N, y, x):
    Np = psf.shape[0]
    return psf[Np // 2 - y:Np // 2 - y + N, Np // 2 - x:Np // 2 - x + N]


def test_clean_gain_one_recovers_separated_sources_exactly():
    """Sources further apart than the PSF, gain 1: each iteration removes one source completely
    (textbook Hogbom), so the model is the source list and the residual is exactly zero."""
    from oracle import clean
    N = 64
    psf = _compact_psf(2 * N)
    src = [(10, 12, 1.0), (30, 40, 0.5), (50, 20, -0.75), (5, 58, 0.25)]
    img = np.zeros((N, N), np.float32)
    for y, x, a in src:
        img += np.float32(a) * _place(psf, N, y, x)
    res, model, comps = clean.hogbom(img, psf, len(src), 1.0)
    assert sorted((y, x, a) for y, x, a in comps) == sorted(src)
    assert np.all(res == 0)
    assert model[10, 12] == 1.0 and model[50, 20] == -0.75 and np.count_nonzero(model) == len(src)


def test_clean_single_source_geometric_decay_and_threshold():
    """One point source: after n iterations the peak residual is a (1 - g)^n and the model holds
    a (1 - (1 - g)^n) at the source; with a threshold t the loop stops after the first n with
    a (1 - g)^n < t."""
    from oracle import clean
    N, a, g = 48, 2.0, 0.2
    psf = _compact_psf(2 * N)
    img = np.float32(a) * _place(psf, N, 20, 27)
    res, model, comps = clean.hogbom(img, psf, 12, g)
    assert len(comps) == 12 and all((y, x) == (20, 27) for y, x, _ in comps)
    assert abs(res[20, 27] - a * (1 - g) ** 12) < 1e-5
    assert abs(model[20, 27] - a * (1 - (1 - g) ** 12)) < 1e-5
    t = 0.3
    _, _, comps = clean.hogbom(img, psf, 100, g, threshold=t)
    assert len(comps) == int(np.ceil(np.log(t / a) / np.log(1 - g)))


def test_clean_search_window_excludes_outside_peaks():
    from oracle import clean
    N = 48
    psf = _compact_psf(2 * N)
    img = 5.0 * _place(psf, N, 5, 5) + 1.0 * _place(psf, N, 30, 30)
    _, model, comps = clean.hogbom(img.astype(np.float32), psf, 1, 1.0, window=(20, 40, 20, 40))
    assert comps == [(30, 30, 1.0)] and model[5, 5] == 0


# ------------------------------------------------------------------------ mosaic phase gradients

def test_per_row_phase_undoes_rephasing_to_pointing_centres():
    """Visibilities of one sky re-phased to per-row pointing centres (the data a mosaic records),
    gridded with those rows' phase gradients, give the grid of the original visibilities gridded
    with none; degridding with the gradients gives the original model visibilities re-phased."""
    from oracle import cf as ocf
    from oracle import index as oindex
    from oracle import ops as oops
    from tests.helpers import mosaic_row_phase, oracle_params
    wl = synth.make_workload("wproj", n_int=6, n_chan=4, grid_n=256, n_wplanes=4, max_support=16, with_vis=True)
    op = oracle_params(wl)
    rp = mosaic_row_phase(wl)
    idx0 = oindex.sample_index(op, wl.uvw_m, wl.freq_hz)
    idx1 = oindex.sample_index(op, wl.uvw_m, wl.freq_hz, row_phase=rp)
    assert np.array_equal(idx0.valid, idx1.valid) and np.array_equal(idx0.p0x, idx1.p0x)
    # the data as recorded at each row's phase centre: V0 exp(-2 pi i (u dl + v dm + w dn)), written
    # out here from the direction cosines of the shift rather than from the oracle's phasor
    sc = wl.freq_hz / synth.C_LIGHT
    u, v, w = (wl.uvw_m[:, k:k + 1] * sc[None, :] for k in range(3))
    dl, dm = rp[:, 0:1], rp[:, 1:2]
    n_shift = np.sqrt(1.0 - dl ** 2 - dm ** 2)
    rephase = np.exp(-2j * np.pi * (u * dl + v * dm + w * (n_shift - 1.0))).reshape(-1, 1)
    V0 = np.asarray(wl.vis, dtype=np.complex128).reshape(-1, wl.n_pol)
    W = np.asarray(wl.weight, dtype=np.float64).reshape(-1, wl.n_pol)
    tabs = ocf.cf_set(op, which=set(np.unique(idx0.cf[idx0.valid]).tolist()))
    buf, off, _ = ocf.flatten_cf_set(op, tabs)
    g0, _ = oops.grid(idx0, buf, off, op.oversampling, op.grid_n, V0, W)
    g1, _ = oops.grid(idx1, buf, off, op.oversampling, op.grid_n, V0 * rephase, W)
    assert np.abs(g1 - g0).max() <= 1e-10 * np.abs(g0).max()
    d0 = oops.degrid(idx0, buf, off, op.oversampling, g0)
    d1 = oops.degrid(idx1, buf, off, op.oversampling, g0)
    assert np.abs(d1 - d0 * rephase).max() <= 1e-10 * np.abs(d0).max()


# ------------------------------------------------------------------------- G-Jones calibration

def _gcal_problem(n_ant=27, n_int=4, C=8, P=4, sol_int=2, sol_chan=4, noise=0.0, seed=6):
    rng = np.random.default_rng(seed)
    a1, a2 = synth.baseline_antennas(n_ant)
    n_bl = len(a1)
    n_ts, n_fs, n_h = -(-n_int // sol_int), -(-C // sol_chan), (1 if P == 1 else 2)
    g = synth.antenna_gains((n_ts, n_fs, n_h, n_ant), seed=seed)
    M = (rng.standard_normal((n_int * n_bl, C, P)) + 1j * rng.standard_normal((n_int * n_bl, C, P))) + 0.5
    V = np.array(M, copy=True)
    hands = [0] if P == 1 else [0, P - 1]
    for t in range(n_int):
        for c in range(C):
            for q, p in enumerate(hands):
                gg = g[t // sol_int, c // sol_chan, q]
                V[t * n_bl:(t + 1) * n_bl, c, p] *= gg[a1] * np.conj(gg[a2])
    if noise:
        V += noise * (rng.standard_normal(V.shape) + 1j * rng.standard_normal(V.shape))
    W = rng.uniform(0.5, 2.0, V.shape)
    return V, M, W, a1, a2, g


def test_gcal_recovers_noise_free_gains():
    """V_ij = g_i conj(g_j) M_ij exactly: Eq. VAvg gives X_ij = g_i conj(g_j), and the iteration of
    Eq. CalUpdateDir / Eq. CalUpdateModel converges to the true gains up to the common phase."""
    from oracle import gcal
    V, M, W, a1, a2, g = _gcal_problem()
    G, its = gcal.gcal(V, M, W, a1, a2, 27, 2, 4, alpha=0.5, delta=1e-13, max_iter=500)
    ref = g * np.conj(g[..., :1]) / np.abs(g[..., :1])
    assert np.abs(G - ref).max() < 1e-9
    assert np.all(its < 500)


def test_gcal_average_of_constant_ratio_and_weights():
    from oracle import gcal
    rng = np.random.default_rng(8)
    n_bl, n_int, C = 6, 3, 5
    M = rng.standard_normal((n_int * n_bl, C, 1)) + 1j * rng.standard_normal((n_int * n_bl, C, 1))
    r = np.exp(1j * rng.uniform(-3, 3, n_bl)) * rng.uniform(0.5, 2, n_bl)
    V = M * np.tile(r, n_int)[:, None, None]
    W = rng.uniform(0.1, 1.0, M.shape)
    W[0, 0, 0] = 0.0   # flagged: skipped
    X, Wt = gcal.average(V, M, W, n_bl, sol_int=n_int, sol_chan=C)
    assert np.allclose(X[0, 0, 0], r, rtol=1e-13, atol=0)
    w = W.reshape(n_int, n_bl, C)
    assert np.allclose(Wt[0, 0, 0], (w * np.abs(M.reshape(n_int, n_bl, C)) ** 2).sum(axis=(0, 2)), rtol=1e-13)


def test_gcal_first_step_closed_form():
    """From g = 1 with alpha = 1, one step of Eq. CalUpdateDir gives g_i = sum_j X_ij w_ij / sum_j w_ij
    (X_ij = conj(X_ji)), written out here as a plain loop."""
    from oracle import gcal
    rng = np.random.default_rng(9)
    n_ant = 4
    a1, a2 = synth.baseline_antennas(n_ant)
    X = rng.standard_normal(len(a1)) + 1j * rng.standard_normal(len(a1))
    Wt = rng.uniform(0.5, 2.0, len(a1))
    g, it = gcal.solve_gains(X, Wt, a1, a2, n_ant, alpha=1.0, delta=0.0, max_iter=1, ref_ant=0)
    want = []
    for i in range(n_ant):
        num = den = 0
        for b in range(len(a1)):
            if a1[b] == i:
                num += X[b] * Wt[b]
                den += Wt[b]
            elif a2[b] == i:
                num += np.conj(X[b]) * Wt[b]
                den += Wt[b]
        want.append(num / den)
    want = np.array(want)
    want = want * np.conj(want[0]) / abs(want[0])
    assert it == 1 and np.allclose(g, want, rtol=1e-14, atol=1e-14)


def test_gcal_lowers_chi2_with_noise():
    """Eq. XChisq, sum w |X_ij - g_i conj(g_j)|^2, falls from the starting gains to the solution."""
    from oracle import gcal
    V, M, W, a1, a2, g = _gcal_problem(noise=0.3, seed=10)
    X, Wt = gcal.average(V, M, W, len(a1), 2, 4)
    for idx in np.ndindex(*X.shape[:3]):
        gs, _ = gcal.solve_gains(X[idx], Wt[idx], a1, a2, 27, 0.5, 1e-12, 500)
        chi = lambda gg: float((Wt[idx] * np.abs(X[idx] - gg[a1] * np.conj(gg[a2])) ** 2).sum())
        assert chi(gs) < 0.1 * chi(np.ones(27))
        gt = g[idx] * np.conj(g[idx][0]) / abs(g[idx][0])
        assert np.abs(gs - gt).max() < 0.05


# ------------------------------------------------------------- full polarisation (Mueller CFs)

def _pol_params(**over):
    kw = dict(grid_n=256, cell_rad=2e-5, oversampling=6, max_support=24, use_w=True, n_wplanes=3,
              w_max_lambda=3e4, use_a=True, n_pa_bins=2, pa_bin_centers=[0.3, -0.9], n_subbands=1,
              subband_freq_hz=[3.0e9], use_pol=True, squint_rad=2.5e-4, leakage=0.05 * np.exp(0.7j),
              mueller_threshold=0.01)
    kw.update(over)
    return cf.CFParams(**kw)


def test_mueller_element_list():
    assert len(cf.mueller_elements(_pol_params())) == 12          # 4 diagonal + 8 with one leakage factor
    assert len(cf.mueller_elements(_pol_params(mueller_threshold=0.002))) == 16
    assert cf.mueller_elements(_pol_params(leakage=0.0)) == [(0, 0), (1, 1), (2, 2), (3, 3)]


def test_mueller_without_squint_or_leakage_is_the_pol_shared_aterm():
    """J = diag(A, A): every diagonal element's screen is A^2, the Airy power pattern of the
    pol-shared A-term, and the element tables equal that CF."""
    p = _pol_params(squint_rad=0.0, leakage=0.0)
    p0 = _pol_params(use_pol=False)
    for e in range(4):
        for ks in range(p.n_signed):
            t = cf.cf_table(p, 1, 0, ks, cf.mueller_elements(p)[e])
            t0 = cf.cf_table(p0, 1, 0, ks)
            assert np.abs(t - t0).max() <= 1e-13 * np.abs(t0).max()


def test_mueller_screens_are_the_jones_kronecker_product():
    """Element (p, q) of the screen is entry (p, q) of kron(J, conj(J)) in the RR, RL, LR, LL
    order (numpy's Kronecker product, not the element formula)."""
    p = _pol_params(mueller_threshold=0.0)
    M = 32
    i = np.arange(M, dtype=np.float64)
    lm = (i - M / 2) * p.grid_n / M * p.cell_rad
    chi = p.pa_bin_centers[0]
    L, Mm = lm[None, :], lm[:, None]
    lr = L * math.cos(chi) + Mm * math.sin(chi)
    mr = -L * math.sin(chi) + Mm * math.cos(chi)
    eps = p.ellipticity
    rr = np.sqrt(((lr - p.squint_rad) / (1 + eps)) ** 2 + (mr / (1 - eps)) ** 2)
    rl = np.sqrt(((lr + p.squint_rad) / (1 + eps)) ** 2 + (mr / (1 - eps)) ** 2)
    ar = cf.airy_voltage(rr, 3.0e9, 25.0)
    al = cf.airy_voltage(rl, 3.0e9, 25.0)
    base = cf.screen(cf.CFParams(grid_n=p.grid_n, cell_rad=p.cell_rad, use_w=True, n_wplanes=3, w_max_lambda=3e4),
                     0, 0, 4, M)
    d = p.leakage
    for y, x in [(3, 5), (16, 16), (20, 9), (31, 0)]:
        J = np.array([[ar[y, x], d * ar[y, x]], [d * al[y, x], al[y, x]]])
        K = np.kron(J, J.conj())
        for e, (pp, qq) in enumerate(cf.mueller_elements(p)):
            s = cf.screen(p, 0, 0, 4, M, (pp, qq))
            assert abs(s[y, x] - base[y, x] * K[pp, qq]) <= 1e-14 * max(1.0, abs(s[y, x]))


def test_mueller_gridding_is_the_adjoint_of_degridding():
    """<G_M V, X> = <V, D_M X> with unit weights for the full Mueller operators."""
    p = _pol_params(grid_n=128, cell_rad=4e-5, max_support=16, oversampling=4)
    wl = synth.make_workload("standard", n_int=3, with_vis=False)
    rng = np.random.default_rng(12)
    uvw = wl.uvw_m * 0.02
    freq = np.array([3.0e9])
    pa = rng.integers(0, 2, uvw.shape[0]).astype(np.int32)
    idx = index.sample_index(p, uvw, freq, pa_bin=pa)
    assert idx.valid.mean() > 0.5
    buf, off, _ = cf.flatten_cf_set(p, cf.cf_set(p))
    n = idx.valid.shape[0]
    V = rng.standard_normal((n, 4)) + 1j * rng.standard_normal((n, 4))
    X = rng.standard_normal((p.grid_n, p.grid_n, 4)) + 1j * rng.standard_normal((p.grid_n, p.grid_n, 4))
    g, _ = ops.grid_mueller(p, idx, buf, off, p.oversampling, p.grid_n, V, np.ones((n, 4)))
    d = ops.degrid_mueller(p, idx, buf, off, p.oversampling, X)
    a, b = np.vdot(g, X), np.vdot(V, d)
    assert abs(a - b) <= 1e-12 * abs(a)
