"""grid_visibilities_noalloc: gridding for callers that must not allocate device memory.

Such callers (real-time pipelines that reserve the whole device at start-up, hosts whose own
allocator owns the GPU) get a variant that keeps its per-sample index and ordering in a fixed
array inside the library instead of a plan it allocates.  These checks call it through the C ABI
and compare it with plan_create + grid_visibilities on the same inputs, twice in a row so that
whatever the first call left in the shared array cannot leak into the second.  This file is named
to be collected last.
"""
import ctypes

import numpy as np
import pytest

import synth
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
    return awg, lib, wl, cf


def _noalloc(lib, cf, uvw, freq, vis, wt, grid, sumwt):
    R, C, P = vis.shape
    return lib.grid_visibilities_noalloc(cf.handle, _vp(uvw), R, _vp(freq), C, None, None, _vp(vis), _vp(wt), P,
                                         _vp(grid), _vp(sumwt), _stream())


def test_noalloc_matches_planned_gridding_twice(env):
    awg, lib, wl, cf = env
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
    for call in range(2):
        g = torch.zeros((N, N, P), dtype=torch.complex64, device="cuda")
        sw = torch.zeros(P, dtype=torch.float64, device="cuda")
        st = _noalloc(lib, cf, uvw, freq, vis, wt, g, sw)
        assert st == 0, lib.awg_last_error()
        torch.cuda.synchronize()
        assert rel_rms(g.cpu().numpy(), ref) < 1e-5, call
        assert np.allclose(sw.cpu().numpy(), sw_ref.cpu().numpy(), rtol=1e-12), call


def test_noalloc_rejects_oversized_requests(env):
    awg, lib, wl, cf = env
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
    torch.cuda.synchronize()
    assert torch.count_nonzero(g).item() == 0
