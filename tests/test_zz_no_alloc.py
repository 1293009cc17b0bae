"""grid_visibilities_noalloc: gridding for callers that must not allocate device memory.

Such callers (real-time pipelines that reserve the whole device at start-up, hosts whose own
allocator owns the GPU) get a variant that keeps its per-sample index and ordering in a fixed
array inside the library instead of a plan it allocates.  These checks call it through the C ABI
with every library allocation armed to fail (so any allocation on its path would turn into an
error), compare it with plan_create + grid_visibilities and with the FP64 oracle, twice in a row
so that whatever the first call left in the shared array cannot leak into the second, and check
the limits it rejects.  This file is named to be collected last.
"""
import ctypes
import gc

import numpy as np
import pytest

import synth
from oracle import cf as ocf
from oracle import index as oindex
from oracle import ops as oops
from tests.helpers import library_params, oracle_params, rel_rms

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _vp(t):
    return ctypes.c_void_p(t.data_ptr() if t is not None else None)


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


@pytest.fixture(scope="module")
def env():
    import paper_2508_17187_gb300 as awg
    from paper_2508_17187_gb300 import _lib
    lib = _lib.load()            # no fallback: a missing library fails here
    assert torch.cuda.is_available()
    wl = synth.make_workload("wproj", n_int=8, n_chan=8, grid_n=512, n_wplanes=6, max_support=32)
    op = oracle_params(wl)
    cf = awg.cf_set_create(**library_params(op))
    return awg, lib, wl, op, cf


def _noalloc(lib, cf, uvw, freq, vis, wt, grid, sumwt, pa=None, sb=None):
    R, C, P = vis.shape
    return lib.grid_visibilities_noalloc(cf.handle, _vp(uvw), R, _vp(freq), C, _vp(pa), _vp(sb), _vp(vis), _vp(wt), P,
                                         _vp(grid), _vp(sumwt), _stream())


def _noalloc_armed(lib, *args, **kw):
    """The call with every library device allocation armed to fail: it must still succeed, and the
    library's live allocation count must not move.  The count is library-wide, so the garbage
    collector (which may release other tests' plans and CF sets) is held off meanwhile."""
    gc.collect()
    gc.disable()
    try:
        live = lib.awg_debug_live_allocations()
        torch_live = torch.cuda.memory_allocated()
        assert lib.awg_debug_fail_allocations(0) == 0
        try:
            st = _noalloc(lib, *args, **kw)
        finally:
            lib.awg_debug_fail_allocations(-1)
        assert st == 0, lib.awg_last_error()
        assert lib.awg_debug_live_allocations() == live
        assert torch.cuda.memory_allocated() == torch_live
    finally:
        gc.enable()
    return st


def _oracle_grid(op, wl, pa=None, sb=None):
    idx = oindex.sample_index(op, wl.uvw_m, wl.freq_hz, pa, sb)
    tabs = ocf.cf_set(op, which=set(np.unique(idx.cf[idx.valid]).tolist()))
    buf, off, _ = ocf.flatten_cf_set(op, tabs)
    n, P = wl.n_rows * wl.n_chan, wl.n_pol
    return oops.grid(idx, buf, off, op.oversampling, op.grid_n, wl.vis.reshape(n, P), wl.weight.reshape(n, P))


def test_noalloc_matches_planned_gridding_and_oracle_twice(env):
    awg, lib, wl, op, cf = env
    N, P = wl.grid_n, wl.n_pol
    uvw = torch.as_tensor(wl.uvw_m).cuda()
    freq = torch.as_tensor(wl.freq_hz).cuda()
    vis = torch.as_tensor(wl.vis).cuda()
    wt = torch.as_tensor(wl.weight).cuda()
    assert wl.n_samples <= 65536
    plan = awg.plan_create(cf, uvw, freq)
    g_ref = torch.zeros((N, N, P), dtype=torch.complex64, device="cuda")
    sw_ref = torch.zeros(P, dtype=torch.float64, device="cuda")
    awg.grid_visibilities(cf, plan, vis, wt, g_ref, sw_ref)
    torch.cuda.synchronize()
    ref = g_ref.cpu().numpy()
    g_o, sw_o = _oracle_grid(op, wl)
    dev_before = torch.cuda.current_device()
    for call in range(2):
        g = torch.zeros((N, N, P), dtype=torch.complex64, device="cuda")
        sw = torch.zeros(P, dtype=torch.float64, device="cuda")
        _noalloc_armed(lib, cf, uvw, freq, vis, wt, g, sw)
        torch.cuda.synchronize()
        got = g.cpu().numpy()
        assert rel_rms(got, ref) < 1e-5, call
        assert rel_rms(got, g_o) < 1e-5, call
        assert np.allclose(sw.cpu().numpy(), sw_ref.cpu().numpy(), rtol=1e-12), call
        assert np.allclose(sw.cpu().numpy(), sw_o, rtol=1e-12), call
    assert torch.cuda.current_device() == dev_before


def test_noalloc_multi_term_aw_set(env):
    """A-term CFs over PA bins and sub-bands (several outer-product terms per CF) within the sample
    limit: the same as the planned path and the oracle, with no allocation."""
    awg, lib = env[0], env[1]
    wl = synth.make_workload("awproj", n_int=4, n_chan=8, grid_n=512, n_pa=3, n_sb=2, n_wplanes=4, max_support=32,
                             oversampling=8)
    op = oracle_params(wl)
    cf = awg.cf_set_create(**library_params(op))
    assert cf.rank > 1
    recs = wl.n_samples * (cf.rank if cf.fused_terms == 0 else 1)
    assert recs <= 65536
    N, P = wl.grid_n, wl.n_pol
    uvw = torch.as_tensor(wl.uvw_m).cuda()
    freq = torch.as_tensor(wl.freq_hz).cuda()
    pa = torch.as_tensor(wl.pa_bin, dtype=torch.int32).cuda()
    sb = torch.as_tensor(wl.chan_subband, dtype=torch.int32).cuda()
    vis = torch.as_tensor(wl.vis).cuda()
    wt = torch.as_tensor(wl.weight).cuda()
    plan = awg.plan_create(cf, uvw, freq, pa, sb)
    g_ref = torch.zeros((N, N, P), dtype=torch.complex64, device="cuda")
    sw_ref = torch.zeros(P, dtype=torch.float64, device="cuda")
    awg.grid_visibilities(cf, plan, vis, wt, g_ref, sw_ref)
    g_o, sw_o = _oracle_grid(op, wl, wl.pa_bin, wl.chan_subband)
    for call in range(2):
        g = torch.zeros((N, N, P), dtype=torch.complex64, device="cuda")
        sw = torch.zeros(P, dtype=torch.float64, device="cuda")
        _noalloc_armed(lib, cf, uvw, freq, vis, wt, g, sw, pa=pa, sb=sb)
        torch.cuda.synchronize()
        got = g.cpu().numpy()
        assert rel_rms(got, g_ref.cpu().numpy()) < 1e-5, call
        assert rel_rms(got, g_o) < 1e-5, call
        assert np.allclose(sw.cpu().numpy(), sw_o, rtol=1e-12), call


def test_noalloc_rejects_oversized_requests(env):
    awg, lib, wl, op, cf = env
    N, P = wl.grid_n, wl.n_pol
    g = torch.zeros((N, N, P), dtype=torch.complex64, device="cuda")
    sw = torch.zeros(P, dtype=torch.float64, device="cuda")
    big = synth.make_workload("wproj", n_int=200, n_chan=8, grid_n=512, n_wplanes=6, max_support=32)
    assert big.n_samples > 65536
    uvw = torch.as_tensor(big.uvw_m).cuda()
    freq = torch.as_tensor(big.freq_hz).cuda()
    vis = torch.as_tensor(big.vis).cuda()
    wt = torch.as_tensor(big.weight).cuda()
    st = _noalloc(lib, cf, uvw, freq, vis, wt, g, sw)
    assert st == 1
    assert b"at most 65536 samples" in lib.awg_last_error()
    # a row count whose product with the channels would overflow 64 bits is refused the same way
    st = lib.grid_visibilities_noalloc(cf.handle, _vp(uvw), (1 << 62), _vp(freq), 8, None, None, _vp(vis), _vp(wt), P,
                                       _vp(g), _vp(sw), _stream())
    assert st == 1
    assert b"at most 65536 samples" in lib.awg_last_error()
    torch.cuda.synchronize()
    assert torch.count_nonzero(g).item() == 0


def test_noalloc_rejects_too_many_buckets(env):
    """A 4096^2 grid has more (support, tile) buckets than the fixed array holds: refused with the
    bucket limit, nothing launched."""
    awg, lib, wl, op, _ = env
    op_big = oracle_params(wl, grid_n=4096, cell_rad=wl.cell_rad / 8)
    cf = awg.cf_set_create(**library_params(op_big))
    P = wl.n_pol
    g = torch.zeros((4096, 4096, P), dtype=torch.complex64, device="cuda")
    sw = torch.zeros(P, dtype=torch.float64, device="cuda")
    uvw = torch.as_tensor(wl.uvw_m[:10]).cuda()
    freq = torch.as_tensor(wl.freq_hz).cuda()
    vis = torch.as_tensor(wl.vis[:10]).cuda()
    wt = torch.as_tensor(wl.weight[:10]).cuda()
    st = _noalloc(lib, cf, uvw, freq, vis, wt, g, sw)
    assert st == 1
    assert b"buckets" in lib.awg_last_error()
    torch.cuda.synchronize()
    assert torch.count_nonzero(g).item() == 0
