"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the same seeded inputs.

Tolerances.  Inputs are FP32 (visibilities, weights, CF values); the oracle sums the same values
in FP64.  Each FP32 product and add carries a relative rounding of at most 2^-24 ~ 6e-8, and a
pixel's sum of n contributions in FP32 has a relative RMS error of order 6e-8 sqrt(n); with
n <= 10^5 that is below 2e-5 in the worst pixel and about 1e-6 over the grid.  The gate used for
whole grids, images and visibility vectors is the 1e-5 relative RMS accuracy target; BF16 CF tables
(8-bit mantissa, 2^-9 relative) get their own, looser gate.  Integer-valued inputs make FP32 sums
exact, and there the comparison is bit for bit.
"""
import dataclasses
import math

import numpy as np
import pytest

import synth
from oracle import cf as ocf
from oracle import image as oimage
from oracle import index as oindex
from oracle import ops as oops
from tests.helpers import inner_half, library_params, oracle_params, rel_rms

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def awg():
    import paper_2508_17187_gb300 as m
    from paper_2508_17187_gb300 import _lib
    _lib.load()          # fails loudly when the library is missing: there is no fallback
    assert torch.cuda.is_available()
    return m


def _dev(a, dtype=None):
    t = torch.as_tensor(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def _run_library(awg, op, uvw, freq, vis, wt, pa_bin=None, chan_sb=None, cf=None, phase_shift=None, flags=0,
                 cf_dtype=0, separable=True):
    """Plan + grid + degrid(grid) through the C ABI; returns host arrays."""
    if cf is None:
        cf = awg.cf_set_create(**library_params(op, cf_dtype, separable))
    R, C = uvw.shape[0], freq.shape[0]
    P = vis.shape[-1]
    N = op.grid_n
    plan = awg.plan_create(cf, _dev(uvw), _dev(freq), None if pa_bin is None else _dev(pa_bin, torch.int32),
                           None if chan_sb is None else _dev(chan_sb, torch.int32), phase_shift=phase_shift)
    g = torch.zeros((N, N, P), dtype=torch.complex128 if flags & awg.AWG_GRID_FP64 else torch.complex64,
                    device="cuda")
    glo = torch.zeros((N, N, P), dtype=torch.complex64, device="cuda") if flags & awg.AWG_GRID_KAHAN else None
    sw = torch.zeros(P, dtype=torch.float64, device="cuda")
    awg.grid_visibilities(cf, plan, _dev(vis.reshape(R, C, P), torch.complex64),
                          _dev(wt.reshape(R, C, P), torch.float32), g, sw, grid_lo=glo, flags=flags)
    gg = g.to(torch.complex128) + (glo.to(torch.complex128) if glo is not None else 0)
    gdeg = gg.to(torch.complex64)
    out = torch.full((R, C, P), complex(7.0, -3.0), dtype=torch.complex64, device="cuda")   # poisoned
    awg.degrid_visibilities(cf, plan, gdeg, out)
    torch.cuda.synchronize()
    stats = plan.stats()
    return dict(grid=gg.cpu().numpy(), sumwt=sw.cpu().numpy(), vis=out.cpu().numpy().reshape(R * C, P),
                grid_used=gdeg.cpu().numpy(), stats=stats, cf=cf, plan=plan)


def _oracle(op, uvw, freq, vis, wt, grid_for_degrid, pa_bin=None, chan_sb=None, phase_shift=None, tables=None):
    idx = oindex.sample_index(op, uvw, freq, pa_bin, chan_sb, phase_shift=phase_shift)
    if tables is None:
        tables = ocf.cf_set(op, which=set(np.unique(idx.cf[idx.valid]).tolist()))
    buf, off, _ = ocf.flatten_cf_set(op, tables)
    n = idx.valid.shape[0]
    P = vis.shape[-1]
    g, sw = oops.grid(idx, buf, off, op.oversampling, op.grid_n, vis.reshape(n, P), wt.reshape(n, P))
    d = oops.degrid(idx, buf, off, op.oversampling, grid_for_degrid.astype(np.complex128))
    return dict(idx=idx, grid=g, sumwt=sw, vis=d)


# ------------------------------------------------------------------------------------------ CF tables

@pytest.mark.parametrize("separable", [True, False])
@pytest.mark.parametrize("mode", ["ps", "wproj", "awproj"])
def test_cf_tables_match_oracle(awg, mode, separable):
    wl = synth.make_workload("standard", n_int=4, with_vis=False)
    over = dict(grid_n=256, cell_rad=2e-5, oversampling=6, max_support=24)
    if mode != "ps":
        over.update(use_w=True, n_wplanes=4, w_max_lambda=4e4)
    if mode == "awproj":
        over.update(use_a=True, n_pa_bins=2, pa_bin_centers=[0.3, -0.9], n_subbands=2,
                    subband_freq_hz=[2.2e9, 3.6e9])
    op = oracle_params(wl, **over)
    cf = awg.cf_set_create(**library_params(op, separable=separable))
    # PS and W CFs are outer products to FP32 precision; A-term CFs are sums of a few
    assert cf.separable == separable
    if separable:
        assert (1 < cf.rank <= 6) if mode == "awproj" else cf.rank == 1
    sup = cf.supports()
    assert np.array_equal(sup, ocf.supports(op))
    for ci in range(op.n_cf):
        pa, rem = divmod(ci, op.n_subbands * op.n_signed)
        sb, ks = divmod(rem, op.n_signed)
        ref = ocf.cf_table(op, pa, sb, ks)
        got = cf.copy_table(ci)
        assert got.shape == ref.shape
        # FP64 build rounded once to FP32 (or FP32 factors and their FP32 products); two
        # different FFT / DFT evaluations of one definition; a fit of several terms stops within
        # 1e-6 of the peak
        tol = 2e-7 if not cf.separable else 3e-7 if cf.rank == 1 else 1.5e-6
        assert np.abs(got - ref).max() <= tol * np.abs(ref).max() + 1e-9, (mode, ci)


# ------------------------------------------------------------------------------------------ exact pins

@pytest.mark.parametrize("separable", [True, False])
def test_delta_cf_is_exact_binning(awg, separable):
    """Support-1 delta CF with integer-valued data: G is direct binning, D direct lookup, bit exact
    (as factors 1 x 1 and as a full table)."""
    wl = synth.make_workload("standard", n_int=30, with_vis=False)
    N = wl.grid_n
    op = oracle_params(wl, oversampling=1, max_support=1, ps_support=1, use_ps=False)
    rng = np.random.default_rng(3)
    n = wl.n_samples
    vis = (rng.integers(-8, 9, n) + 1j * rng.integers(-8, 9, n)).astype(np.complex64).reshape(-1, 1)
    wt = rng.integers(0, 4, n).astype(np.float32).reshape(-1, 1)
    cf = awg.cf_set_create_from_table([1], np.ones(4, dtype=np.complex64), **library_params(op, separable=separable))
    assert cf.separable == separable
    res = _run_library(awg, op, wl.uvw_m, wl.freq_hz, vis, wt, cf=cf)
    sc = wl.freq_hz / synth.C_LIGHT
    u = (wl.uvw_m[:, 0:1] * sc).reshape(-1)
    v = (wl.uvw_m[:, 1:2] * sc).reshape(-1)
    ix = np.floor(u * (N * wl.cell_rad) + N // 2 + 0.5).astype(np.int64)
    iy = np.floor(v * (N * wl.cell_rad) + N // 2 + 0.5).astype(np.int64)
    ref = np.zeros((N, N), dtype=np.complex128)
    np.add.at(ref, (iy, ix), wt[:, 0].astype(np.float64) * vis[:, 0])
    assert np.array_equal(res["grid"][:, :, 0], ref)
    assert res["sumwt"][0] == wt.astype(np.float64).sum()
    assert np.array_equal(res["vis"][:, 0], res["grid_used"][iy, ix, 0])
    assert res["stats"][:2] == (n, 0)


# ------------------------------------------------------------------------------------------ parity

@pytest.mark.parametrize("separable", [True, False])
def test_standard_grid_degrid_parity(awg, separable):
    wl = synth.make_workload("standard", n_int=40)
    op = oracle_params(wl)
    vis = wl.vis.reshape(-1, 1)
    wt = wl.weight.reshape(-1, 1)
    res = _run_library(awg, op, wl.uvw_m, wl.freq_hz, vis, wt, separable=separable)
    orc = _oracle(op, wl.uvw_m, wl.freq_hz, vis, wt, res["grid_used"])
    assert res["stats"][0] == int(orc["idx"].valid.sum())
    assert rel_rms(res["grid"], orc["grid"]) < 1e-5
    assert np.allclose(res["sumwt"], orc["sumwt"], rtol=1e-12)
    img = oimage.dirty_image(res["grid"], res["sumwt"], wl.ps_support)
    img_o = oimage.dirty_image(orc["grid"], orc["sumwt"], wl.ps_support)
    assert rel_rms(inner_half(img), inner_half(img_o)) < 1e-5
    assert rel_rms(res["vis"], orc["vis"]) < 1e-5


@pytest.mark.parametrize("separable", [True, False])
def test_wproj_parity_several_tiles_ragged(awg, separable):
    """W-projection, 4 pols, OS 20, supports 8..64 over 8 signed planes: every CF class, many tiles,
    ragged work items; separable (factor) and full-table CF storage."""
    wl = synth.make_workload("wproj", n_int=24, n_chan=8, grid_n=1024)
    op = oracle_params(wl, n_wplanes=8)
    vis = wl.vis.reshape(-1, 4)
    wt = wl.weight.reshape(-1, 4)
    res = _run_library(awg, op, wl.uvw_m, wl.freq_hz, vis, wt, separable=separable)
    assert res["cf"].separable == separable
    orc = _oracle(op, wl.uvw_m, wl.freq_hz, vis, wt, res["grid_used"])
    assert res["stats"][0] == int(orc["idx"].valid.sum())
    assert res["stats"][1] == int((~orc["idx"].valid).sum())
    assert res["stats"][2] == int((orc["idx"].support[orc["idx"].valid].astype(np.int64) ** 2).sum())
    assert rel_rms(res["grid"], orc["grid"]) < 1e-5
    img = oimage.dirty_image(res["grid"], res["sumwt"], wl.ps_support)
    img_o = oimage.dirty_image(orc["grid"], orc["sumwt"], wl.ps_support)
    assert rel_rms(inner_half(img), inner_half(img_o)) < 1e-5
    assert rel_rms(res["vis"], orc["vis"]) < 1e-5
    dropped = ~orc["idx"].valid
    assert np.all(res["vis"][dropped] == 0)


@pytest.mark.parametrize("separable", [True, False])
def test_awproj_parity(awg, separable):
    """A-term CFs over PA bins and sub-bands plus W planes (Tab. AWP-CFSETUP, AW-Projection), stored
    as sums of outer products (one plan record per sample and term) or as full tables."""
    wl = synth.make_workload("awproj", n_int=12, n_chan=8, grid_n=512, n_pa=3, n_sb=2, n_wplanes=4, max_support=32,
                             oversampling=8)
    op = oracle_params(wl)
    vis = wl.vis.reshape(-1, 4)
    wt = wl.weight.reshape(-1, 4)
    res = _run_library(awg, op, wl.uvw_m, wl.freq_hz, vis, wt, pa_bin=wl.pa_bin, chan_sb=wl.chan_subband,
                       separable=separable)
    assert res["cf"].separable == separable
    if separable:
        assert 1 < res["cf"].rank <= 6
    orc = _oracle(op, wl.uvw_m, wl.freq_hz, vis, wt, res["grid_used"], pa_bin=wl.pa_bin, chan_sb=wl.chan_subband)
    assert res["stats"][0] == int(orc["idx"].valid.sum())
    assert rel_rms(res["grid"], orc["grid"]) < 1e-5
    # each sample's weight counted once, whatever the number of terms
    assert np.allclose(res["sumwt"], orc["sumwt"], rtol=1e-12)
    assert rel_rms(res["vis"], orc["vis"]) < 1e-5
    assert np.all(res["vis"][~orc["idx"].valid] == 0)


@pytest.mark.parametrize("fused", [True, False])
def test_mueller_full_polarisation_parity(awg, fused):
    """Sparse Mueller matrix of A-term CFs (feed squint and complex leakage, 12 of 16 elements kept):
    CF tables, gridding (pol q from conj(CF_pq) w_p V_p), weight sums and degridding against the
    oracle.  fused: W-projection supports 8..32 (the 4-pol base passes with pol mixing); not fused:
    no W term and support 20, which has no exact-support kernel (one single-pol pass per element)."""
    if fused:
        wl = synth.make_workload("awproj", n_int=10, n_chan=8, grid_n=512, n_pa=3, n_sb=2, n_wplanes=4,
                                 max_support=32, oversampling=8)
        op = oracle_params(wl, use_pol=True, squint_rad=3e-4, leakage=0.04 * np.exp(0.9j), mueller_threshold=0.01)
    else:
        wl = synth.make_workload("awproj", n_int=10, n_chan=8, grid_n=512, n_pa=3, n_sb=2, n_wplanes=4,
                                 max_support=20, oversampling=8)
        op = oracle_params(wl, use_pol=True, squint_rad=3e-4, leakage=0.04 * np.exp(0.9j), mueller_threshold=0.01)
        op = dataclasses.replace(op, use_w=False)
    cf = awg.cf_set_create(**library_params(op))
    assert cf.mueller() == ocf.mueller_elements(op) and len(cf.mueller()) == 12
    assert cf.separable and cf.rank >= 1
    assert (cf.fused_terms > 0) == fused
    assert cf.n_cf == op.n_cf
    # a diagonal and a leakage element table
    for e in (0, 1):
        ci = e * op.n_base + op.cf_index(1, 1, op.n_signed - 1)
        ref = ocf.cf_table(op, 1, 1, op.n_signed - 1, ocf.mueller_elements(op)[e])
        assert np.abs(cf.copy_table(ci) - ref).max() <= 1.5e-6 * np.abs(ref).max() + 1e-9
    R, C, N = wl.n_rows, wl.n_chan, wl.grid_n
    vis = wl.vis.reshape(-1, 4)
    wt = wl.weight.reshape(-1, 4)
    plan = awg.plan_create(cf, _dev(wl.uvw_m), _dev(wl.freq_hz), _dev(wl.pa_bin, torch.int32),
                           _dev(wl.chan_subband, torch.int32))
    g = torch.zeros((N, N, 4), dtype=torch.complex64, device="cuda")
    sw = torch.zeros(4, dtype=torch.float64, device="cuda")
    awg.grid_visibilities(cf, plan, _dev(vis.reshape(R, C, 4), torch.complex64), _dev(wt.reshape(R, C, 4), torch.float32),
                          g, sw)
    out = torch.full((R, C, 4), complex(5.0, 1.0), dtype=torch.complex64, device="cuda")
    awg.degrid_visibilities(cf, plan, g, out)
    idx = oindex.sample_index(op, wl.uvw_m, wl.freq_hz, wl.pa_bin, wl.chan_subband)
    buf, off, _ = ocf.flatten_cf_set(op, ocf.cf_set(op))
    g_o, sw_o = oops.grid_mueller(op, idx, buf, off, op.oversampling, N, vis.astype(np.complex128),
                                  wt.astype(np.float64))
    assert rel_rms(g.cpu().numpy(), g_o) < 1e-5
    assert np.allclose(sw.cpu().numpy(), sw_o, rtol=1e-12)
    d_o = oops.degrid_mueller(op, idx, buf, off, op.oversampling, g.cpu().numpy().astype(np.complex128))
    assert rel_rms(out.cpu().numpy().reshape(-1, 4), d_o) < 1e-5
    assert np.all(out.cpu().numpy().reshape(-1, 4)[~idx.valid] == 0)


def _random_tables_case(awg, P, rank1, config=0, terms=1, sups=None):
    sups = sups or [1, 3, 7, 8, 9, 15, 16, 17, 24, 25, 31, 32, 33, 40, 48, 49, 56, 63, 64]
    wl = synth.make_workload("standard", n_int=16, n_chan=3, f_lo=2.8e9, f_hi=3.2e9, with_vis=False)
    N = 384
    OS = 3
    op = ocf.CFParams(grid_n=N, cell_rad=wl.cell_rad * 512 / N * 0.45, oversampling=OS, ps_support=1, use_ps=False,
                      n_pa_bins=len(sups), max_support=64)
    rng = np.random.default_rng(100 + P + (10 if rank1 else 0))

    def cplx(*shape):
        return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)

    flat = []
    for S in sups:
        if rank1:
            # a sum of `terms` outer products fy[oy][ty] fx[ox][tx]: stored as factors by the library
            # (term k scaled by 0.3^k, so that the library's term-by-term fit separates them)
            t = sum(0.3 ** k * cplx(OS + 1, S)[:, None, :, None] * cplx(OS + 1, S)[None, :, None, :]
                    for k in range(terms))
        else:
            t = cplx(OS + 1, OS + 1, S, S)
        flat.append(t.astype(np.complex64).astype(np.complex128).reshape(-1))
    R, C = wl.n_rows, wl.n_chan
    pa_bin = rng.integers(0, len(sups), R).astype(np.int32)
    idx = oindex.sample_index(op, wl.uvw_m, wl.freq_hz, pa_bin=pa_bin, supports=sups)
    assert idx.valid.mean() > 0.5
    assert set(np.unique(idx.support[idx.valid]).tolist()) == set(sups)
    offs = np.zeros(len(sups), dtype=np.int64)
    offs[1:] = np.cumsum([(OS + 1) ** 2 * s * s for s in sups])[:-1]
    buf = np.concatenate(flat)
    n = R * C
    V = (rng.standard_normal((n, P)) + 1j * rng.standard_normal((n, P))).astype(np.complex64)
    W = rng.uniform(0.5, 2.0, (n, P)).astype(np.float32)
    cfset = awg.cf_set_create_from_table(sups, buf.astype(np.complex64), grid_n=N, cell_rad=op.cell_rad,
                                         oversampling=OS, n_pa_bins=len(sups), separable=True)
    assert cfset.separable == rank1
    if rank1:
        assert cfset.rank == terms
        assert cfset.fused_terms == (terms if terms > 1 and sups is not None else 0)
    if config:
        for S in sups:
            if S % 8 == 0:
                cfset.choose(S, config)
    res = _run_library(awg, op, wl.uvw_m, wl.freq_hz, V, W, pa_bin=pa_bin, cf=cfset)
    g_o, sw_o = oops.grid(idx, buf, offs, OS, N, V.astype(np.complex128), W.astype(np.float64))
    assert rel_rms(res["grid"], g_o) < 1e-5
    assert np.allclose(res["sumwt"], sw_o, rtol=1e-12)
    d_o = oops.degrid(idx, buf, offs, OS, res["grid_used"].astype(np.complex128))
    assert rel_rms(res["vis"], d_o) < 1e-5
    # per-support check: every kernel (exact-support or class) is right on its own samples
    for S in sups:
        m = idx.valid & (idx.support == S)
        assert rel_rms(res["vis"][m], d_o[m]) < 1e-5, S
    # adjoint on the GPU with unit weights: <G V, X> = <V, D X>
    X = (rng.standard_normal((N, N, P)) + 1j * rng.standard_normal((N, N, P))).astype(np.complex64)
    plan = res["plan"]
    g = torch.zeros((N, N, P), dtype=torch.complex64, device="cuda")
    sw = torch.zeros(P, dtype=torch.float64, device="cuda")
    awg.grid_visibilities(cfset, plan, _dev(V.reshape(R, C, P)), torch.ones((R, C, P), device="cuda"), g, sw)
    dx = torch.zeros((R, C, P), dtype=torch.complex64, device="cuda")
    awg.degrid_visibilities(cfset, plan, _dev(X), dx)
    a = np.vdot(g.cpu().numpy().astype(np.complex128), X.astype(np.complex128))
    b = np.vdot(V.reshape(R, C, P).astype(np.complex128), dx.cpu().numpy().astype(np.complex128))
    assert abs(a - b) <= 1e-5 * abs(a)
    plan.check()   # no bounded wait gave up


@pytest.mark.parametrize("P", [1, 2, 4])
def test_every_support_class_random_tables(awg, P):
    """Random (non-symmetric, full-rank) tables with supports 1..64 spread over all kernel classes;
    CF chosen per row through the PA-bin index.  Also checks <G V, X> = <V, D X> on the GPU."""
    _random_tables_case(awg, P, rank1=False)


@pytest.mark.parametrize("terms", [2, 3, 4])
@pytest.mark.parametrize("P", [1, 2, 4])
def test_fused_kernels_random_low_rank_tables(awg, P, terms):
    """Random tables of 2, 3 and 4 outer-product terms on the exact supports: the fused kernels
    (one record per sample, the CF formed per tap from its terms) against the oracle."""
    _random_tables_case(awg, P, rank1=True, terms=terms, sups=[8, 16, 24, 32, 40, 48, 56, 64])


@pytest.mark.parametrize("config", [0, 1, 2, 3])
@pytest.mark.parametrize("P", [1, 2, 4])
def test_every_support_separable_random_factors(awg, P, config):
    """Random outer-product tables with the same supports: the separable path, every exact-support
    kernel (8, 16, ..., 64) in its four compiled configurations (2: the warp-specialised kernels,
    3: tensor-core gridding) and every class kernel for the supports in between."""
    _random_tables_case(awg, P, rank1=True, config=config)


@pytest.mark.parametrize("separable", [True, False])
def test_phase_shift_parity(awg, separable):
    """The phase-gradient term of Eq. CIJ: G multiplies by the phasor, D by its conjugate."""
    wl = synth.make_workload("standard", n_int=30)
    op = oracle_params(wl)
    shift = (40 * wl.cell_rad, -25 * wl.cell_rad)
    vis = wl.vis.reshape(-1, 1)
    wt = wl.weight.reshape(-1, 1)
    res = _run_library(awg, op, wl.uvw_m, wl.freq_hz, vis, wt, phase_shift=shift, separable=separable)
    orc = _oracle(op, wl.uvw_m, wl.freq_hz, vis, wt, res["grid_used"], phase_shift=shift)
    assert rel_rms(res["grid"], orc["grid"]) < 2e-5
    assert rel_rms(res["vis"], orc["vis"]) < 2e-5


@pytest.mark.parametrize("separable", [True, False])
def test_mosaic_row_phase_parity(awg, separable):
    """Per-row phase centres (mosaic pointings plus pointing offsets, Tab. AWPSETUP-MOSAICKING):
    against the oracle, and switching back to no shift restores the plain result."""
    from tests.helpers import mosaic_row_phase
    wl = synth.make_workload("wproj", n_int=12, n_chan=6, grid_n=512, n_wplanes=6, max_support=32)
    op = oracle_params(wl)
    rp = mosaic_row_phase(wl)
    cf = awg.cf_set_create(**library_params(op, separable=separable))
    R, C, P, N = wl.n_rows, wl.n_chan, wl.n_pol, wl.grid_n
    uvw, freq = _dev(wl.uvw_m), _dev(wl.freq_hz)
    plan = awg.plan_create(cf, uvw, freq)
    plan.set_row_phase(_dev(rp), uvw, freq)
    vis = _dev(wl.vis.reshape(R, C, P), torch.complex64)
    wt = _dev(wl.weight.reshape(R, C, P), torch.float32)
    g = torch.zeros((N, N, P), dtype=torch.complex64, device="cuda")
    sw = torch.zeros(P, dtype=torch.float64, device="cuda")
    awg.grid_visibilities(cf, plan, vis, wt, g, sw)
    out = torch.empty_like(vis)
    awg.degrid_visibilities(cf, plan, g, out)
    idx = oindex.sample_index(op, wl.uvw_m, wl.freq_hz, row_phase=rp)
    buf, off, _ = ocf.flatten_cf_set(op, ocf.cf_set(op, which=set(np.unique(idx.cf[idx.valid]).tolist())))
    g_o, _ = oops.grid(idx, buf, off, op.oversampling, N, wl.vis.reshape(-1, P).astype(np.complex128),
                       wl.weight.reshape(-1, P).astype(np.float64))
    assert rel_rms(g.cpu().numpy(), g_o) < 2e-5
    d_o = oops.degrid(idx, buf, off, op.oversampling, g.cpu().numpy().astype(np.complex128))
    assert rel_rms(out.cpu().numpy().reshape(-1, P), d_o) < 2e-5
    # back to no shift: the plain operator
    plan.set_row_phase(None, uvw, freq)
    g2 = torch.zeros_like(g)
    awg.grid_visibilities(cf, plan, vis, wt, g2, sw)
    idx0 = oindex.sample_index(op, wl.uvw_m, wl.freq_hz)
    g0, _ = oops.grid(idx0, buf, off, op.oversampling, N, wl.vis.reshape(-1, P).astype(np.complex128),
                      wl.weight.reshape(-1, P).astype(np.float64))
    assert rel_rms(g2.cpu().numpy(), g0) < 1e-5


@pytest.mark.parametrize("separable", [True, False])
@pytest.mark.parametrize("flags", ["kahan", "fp64"])
def test_precision_variants(awg, flags, separable):
    wl = synth.make_workload("wproj", n_int=16, n_chan=6, grid_n=512, n_wplanes=6, max_support=32)
    op = oracle_params(wl)
    vis = wl.vis.reshape(-1, 4)
    wt = wl.weight.reshape(-1, 4)
    f = awg.AWG_GRID_KAHAN if flags == "kahan" else awg.AWG_GRID_FP64
    res = _run_library(awg, op, wl.uvw_m, wl.freq_hz, vis, wt, flags=f, separable=separable)
    plain = _run_library(awg, op, wl.uvw_m, wl.freq_hz, vis, wt, cf=res["cf"])
    orc = _oracle(op, wl.uvw_m, wl.freq_hz, vis, wt, res["grid_used"])
    e_var = rel_rms(res["grid"], orc["grid"])
    e_plain = rel_rms(plain["grid"], orc["grid"])
    assert e_var < 1e-5 and e_plain < 1e-5
    # the sample order inside a work item is not fixed, so both errors carry run-to-run noise
    assert e_var <= e_plain * 1.5


def test_bf16_cf_storage(awg):
    """BF16 CF tables: exact against an oracle fed the same rounded tables; the error against the
    FP32 tables is reported by the precision sweep, here only bounded by the BF16 step."""
    wl = synth.make_workload("wproj", n_int=16, n_chan=6, grid_n=512, n_wplanes=6, max_support=32)
    op = oracle_params(wl)
    vis = wl.vis.reshape(-1, 4)
    wt = wl.weight.reshape(-1, 4)
    res = _run_library(awg, op, wl.uvw_m, wl.freq_hz, vis, wt, cf_dtype=1)
    tables = {ci: res["cf"].copy_table(ci).astype(np.complex128) for ci in range(op.n_cf)}
    orc = _oracle(op, wl.uvw_m, wl.freq_hz, vis, wt, res["grid_used"], tables=tables)
    assert rel_rms(res["grid"], orc["grid"]) < 1e-5
    assert rel_rms(res["vis"], orc["vis"]) < 1e-5
    orc32 = _oracle(op, wl.uvw_m, wl.freq_hz, vis, wt, res["grid_used"])
    assert rel_rms(res["grid"], orc32["grid"]) < 2e-2


# ------------------------------------------------------------------------------------------ edge cases

def test_empty_and_all_dropped(awg):
    wl = synth.make_workload("standard", n_int=2)
    op = oracle_params(wl)
    cf = awg.cf_set_create(**library_params(op))
    N = op.grid_n
    g = torch.zeros((N, N, 1), dtype=torch.complex64, device="cuda")
    sw = torch.zeros(1, dtype=torch.float64, device="cuda")
    empty = awg.plan_create(cf, torch.zeros((0, 3), dtype=torch.float64, device="cuda"), _dev(wl.freq_hz))
    awg.grid_visibilities(cf, empty, torch.zeros((0, 1, 1), dtype=torch.complex64, device="cuda"),
                          torch.zeros((0, 1, 1), dtype=torch.float32, device="cuda"), g, sw)
    assert empty.stats() == (0, 0, 0)
    far = wl.uvw_m * 1e4
    plan = awg.plan_create(cf, _dev(far), _dev(wl.freq_hz))
    awg.grid_visibilities(cf, plan, _dev(wl.vis), _dev(wl.weight), g, sw)
    out = torch.full(tuple(wl.vis.shape), complex(1.0, 1.0), dtype=torch.complex64, device="cuda")
    awg.degrid_visibilities(cf, plan, g, out)
    torch.cuda.synchronize()
    assert plan.stats()[:2] == (0, wl.n_samples)
    assert torch.count_nonzero(g).item() == 0 and sw.item() == 0.0
    assert torch.count_nonzero(out).item() == 0


def test_argument_errors(awg):
    wl = synth.make_workload("standard", n_int=2)
    op = oracle_params(wl)
    cf = awg.cf_set_create(**library_params(op))
    plan = awg.plan_create(cf, _dev(wl.uvw_m), _dev(wl.freq_hz))
    N = op.grid_n
    g = torch.zeros((N, N, 1), dtype=torch.complex64, device="cuda")
    sw = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(awg.AwgError, match="INVALID_ARG"):
        awg.grid_visibilities(cf, plan, _dev(wl.vis), _dev(wl.weight), g, sw, flags=awg.AWG_GRID_KAHAN)
    with pytest.raises(awg.AwgError, match="UNSUPPORTED"):
        awg.cf_set_create(**library_params(oracle_params(wl, max_support=65)))
    with pytest.raises(awg.AwgError, match="INVALID_ARG"):
        awg.cf_set_create(**library_params(oracle_params(wl, use_w=True, n_wplanes=1)))


def test_plain_fp64_baseline_parity(awg):
    """The plain FP64 per-channel baseline matches the oracle (FP64 sums of the FP32 tables)."""
    import ctypes
    from paper_2508_17187_gb300 import _lib
    lib = _lib.load()
    wl = synth.make_workload("wproj", n_int=10, n_chan=4, grid_n=512, n_wplanes=6, max_support=32)
    op = oracle_params(wl)
    cf = awg.cf_set_create(**library_params(op, separable=False))
    N, P, R, C = wl.grid_n, wl.n_pol, wl.n_rows, wl.n_chan
    uvw = _dev(wl.uvw_m)
    vis = _dev(wl.vis)
    wt = _dev(wl.weight)
    freq = np.ascontiguousarray(wl.freq_hz)
    g = torch.zeros((N, N, P), dtype=torch.complex128, device="cuda")
    sw = torch.zeros(P, dtype=torch.float64, device="cuda")
    vp = lambda t: ctypes.c_void_p(t.data_ptr())
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    fp = freq.ctypes.data_as(ctypes.c_void_p)
    assert lib.grid_visibilities_plain_fp64(cf.handle, vp(uvw), R, fp, C, 0, C, None, None, vp(vis), vp(wt), P,
                                            vp(g), vp(sw), st) == 0
    out = torch.zeros((R, C, P), dtype=torch.complex64, device="cuda")
    assert lib.degrid_visibilities_plain_fp64(cf.handle, vp(uvw), R, fp, C, 0, C, None, None, vp(g), vp(out), P,
                                              st) == 0
    torch.cuda.synchronize()
    tables = {ci: cf.copy_table(ci).astype(np.complex128) for ci in range(op.n_cf)}
    orc = _oracle(op, wl.uvw_m, wl.freq_hz, wl.vis.reshape(-1, P), wl.weight.reshape(-1, P), g.cpu().numpy(),
                  tables=tables)
    assert rel_rms(g.cpu().numpy(), orc["grid"]) < 1e-12
    assert np.allclose(sw.cpu().numpy(), orc["sumwt"], rtol=1e-12)
    assert rel_rms(out.cpu().numpy().reshape(-1, P), orc["vis"]) < 1e-6
    sep = awg.cf_set_create(**library_params(op))
    assert lib.grid_visibilities_plain_fp64(sep.handle, vp(uvw), R, fp, C, 0, C, None, None, vp(vis), vp(wt), P,
                                            vp(g), vp(sw), st) == 2
