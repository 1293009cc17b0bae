"""AWG_DEGRID_SUBTRACT: degridding that forms the residual V - D(grid) of Eq. ResIm in place, checked
against V minus the plain degridding of the same grid on every degridding path:
* the four configurations of the exact-support separable kernels (W-projection);
* full CF tables;
* multi-term A-term sets on the fused kernels and as expanded records (per-term sums);
* full polarisation on the fused base passes and on the per-element passes.

A sample's model value is formed the same way in both modes, and the subtraction is one FP32
operation either way, so the two agree bit for bit wherever each output is written once. The
per-element full-polarisation passes add (or subtract) one element at a time, so there the two
orders of FP32 rounding differ and the check is to FP32 rounding. Dropped samples keep their input.
"""
import dataclasses

import numpy as np
import pytest

import synth
from oracle import index as oindex
from tests.helpers import library_params, oracle_params

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# image cells 1.5 times the workload's: the grid then covers less of the uv plane and the longest
# baselines' samples are dropped (0.4-1% of them), so that both kinds of sample are checked
_COARSE = 1.5


@pytest.fixture(scope="module")
def awg():
    import paper_2508_17187_gb300 as m
    from paper_2508_17187_gb300 import _lib
    _lib.load()
    assert torch.cuda.is_available()
    return m


def _dev(a, dtype=None):
    t = torch.as_tensor(np.ascontiguousarray(a))
    return (t.to(dtype) if dtype is not None else t).cuda()


def _check(awg, wl, op, cf, exact=True):
    R, C, P, N = wl.n_rows, wl.n_chan, wl.vis.shape[-1], wl.grid_n
    pa = _dev(wl.pa_bin, torch.int32) if wl.use_a else None
    sb = _dev(wl.chan_subband, torch.int32) if wl.use_a else None
    plan = awg.plan_create(cf, _dev(wl.uvw_m), _dev(wl.freq_hz), pa, sb)
    gen = torch.Generator(device="cuda").manual_seed(7)
    grid = torch.complex(torch.randn((N, N, P), device="cuda", generator=gen),
                         torch.randn((N, N, P), device="cuda", generator=gen)).to(torch.complex64)
    vis = _dev(wl.vis.reshape(R, C, P), torch.complex64)
    model = torch.empty_like(vis)
    awg.degrid_visibilities(cf, plan, grid, model)
    res = vis.clone()
    awg.degrid_visibilities(cf, plan, grid, res, subtract=True)
    torch.cuda.synchronize()
    idx = oindex.sample_index(op, wl.uvw_m, wl.freq_hz, wl.pa_bin if wl.use_a else None,
                              wl.chan_subband if wl.use_a else None)
    kept = torch.as_tensor(idx.valid.reshape(R, C)).cuda()
    assert 0 < int(kept.sum()) < R * C   # both kinds present
    want = torch.where(kept[..., None], vis - model, vis)
    if exact:
        assert torch.equal(res, want)
    else:
        err = (res - want).abs().pow(2).sum().sqrt() / (vis.abs().pow(2).sum() + model.abs().pow(2).sum()).sqrt()
        assert float(err) < 1e-6
        assert torch.equal(res[~kept], vis[~kept])


@pytest.mark.parametrize("config", [0, 1, 2, 3])
def test_subtract_wproj_every_configuration(awg, config):
    wl = synth.make_workload("wproj", n_int=24, n_chan=8, grid_n=1024)
    op = oracle_params(wl, n_wplanes=8, cell_rad=wl.cell_rad * _COARSE)
    cf = awg.cf_set_create(**library_params(op))
    for S in sorted(set(int(s) for s in cf.supports())):
        if S % 8 == 0:
            cf.choose(S, config)
    _check(awg, wl, op, cf)


def test_subtract_full_tables(awg):
    wl = synth.make_workload("wproj", n_int=12, n_chan=8, grid_n=512)
    op = oracle_params(wl, n_wplanes=4, max_support=24, cell_rad=wl.cell_rad * _COARSE)
    cf = awg.cf_set_create(**library_params(op, separable=False))
    assert not cf.separable
    _check(awg, wl, op, cf)


@pytest.mark.parametrize("fused", [True, False])
def test_subtract_multi_term_aw(awg, fused):
    """fused: supports 8..32 with exact kernels (one record per sample); expanded: no W term and
    support 20 (one record per term, summed by k_sum_terms)."""
    wl = synth.make_workload("awproj", n_int=10, n_chan=8, grid_n=512, n_pa=3, n_sb=2, n_wplanes=4,
                             max_support=32 if fused else 20, oversampling=8)
    op = oracle_params(wl, cell_rad=wl.cell_rad * _COARSE)
    if not fused:
        op = dataclasses.replace(op, use_w=False)
    cf = awg.cf_set_create(**library_params(op))
    assert cf.rank > 1 and (cf.fused_terms > 0) == fused
    _check(awg, wl, op, cf)


@pytest.mark.parametrize("fused", [True, False])
def test_subtract_full_polarisation(awg, fused):
    wl = synth.make_workload("awproj", n_int=10, n_chan=8, grid_n=512, n_pa=3, n_sb=2, n_wplanes=4,
                             max_support=32 if fused else 20, oversampling=8)
    op = oracle_params(wl, use_pol=True, squint_rad=3e-4, leakage=0.04 * np.exp(0.9j), mueller_threshold=0.01,
                       cell_rad=wl.cell_rad * _COARSE)
    if not fused:
        op = dataclasses.replace(op, use_w=False)
    cf = awg.cf_set_create(**library_params(op))
    assert (cf.fused_terms > 0) == fused
    _check(awg, wl, op, cf, exact=fused)


def test_subtract_rejects_unknown_flags(awg):
    from paper_2508_17187_gb300 import _lib
    wl = synth.make_workload("standard", n_int=4)
    op = oracle_params(wl)
    cf = awg.cf_set_create(**library_params(op))
    plan = awg.plan_create(cf, _dev(wl.uvw_m), _dev(wl.freq_hz))
    N, P = wl.grid_n, wl.vis.shape[-1]
    g = torch.zeros((N, N, P), dtype=torch.complex64, device="cuda")
    out = torch.zeros((wl.n_rows, wl.n_chan, P), dtype=torch.complex64, device="cuda")
    lib = _lib.load()
    import ctypes
    st = lib.degrid_visibilities(cf.handle, plan.handle, ctypes.c_void_p(g.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                 P, 2, None)
    assert st == 1   # AWG_ERR_INVALID_ARG
