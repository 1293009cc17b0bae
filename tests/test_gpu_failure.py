"""Failure detection without a GPU fault: the library's allocation hook makes the n-th device
allocation fail as out of memory (host side; the driver is never asked), for every n a call
makes.  Each failing call must return AWG_ERR_OOM and free everything it had allocated (the live
allocation count returns to its value before the call), and the context stays usable: the next
call without the hook succeeds and computes."""
import numpy as np
import pytest

import synth
from tests.helpers import library_params, oracle_params

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

AWG_ERR_OOM = 3


@pytest.fixture
def hook():
    from paper_2508_17187_gb300 import _lib
    lib = _lib.load()
    yield lib
    lib.awg_debug_fail_allocations(-1)


def _every_failure(lib, call, holds=True, max_allocs=64):
    """Run call() with the n-th allocation failing for n = 0, 1, ... until it succeeds; returns the
    number of allocations the call makes.  holds: the successful call keeps them (a CF set or a
    plan, closed here), else it frees them itself."""
    from paper_2508_17187_gb300._lib import AwgError
    for n in range(max_allocs):
        base = lib.awg_debug_live_allocations()
        lib.awg_debug_fail_allocations(n)
        try:
            obj = call()
        except AwgError as e:
            assert e.status == AWG_ERR_OOM, e
            assert lib.awg_debug_live_allocations() == base, f"allocation {n}: leaked"
            continue
        finally:
            lib.awg_debug_fail_allocations(-1)
        made = lib.awg_debug_live_allocations() - base
        assert made == (n if holds else 0), (made, n)   # it failed at every earlier allocation
        if obj is not None:
            obj.close()
        assert lib.awg_debug_live_allocations() == base
        return n
    raise AssertionError("the call never succeeded")


def test_cf_set_create_and_plan_create_fail_cleanly(hook):
    import paper_2508_17187_gb300 as awg
    wl = synth.make_workload("awproj", n_int=6, n_chan=8, grid_n=512, n_pa=3, n_sb=2, n_wplanes=4, max_support=32,
                             oversampling=8, with_vis=True)
    op = oracle_params(wl, use_pol=True, squint_rad=3e-4, leakage=0.04 * np.exp(0.9j), mueller_threshold=0.01)
    n_cf = _every_failure(hook, lambda: awg.cf_set_create(**library_params(op)))
    assert n_cf >= 5   # factors, offsets, supports, taper, mixing matrices
    n_tab = _every_failure(hook, lambda: awg.cf_set_create(**library_params(oracle_params(
        synth.make_workload("standard", n_int=4, with_vis=False)), separable=False)))
    assert n_tab >= 4
    cf = awg.cf_set_create(**library_params(op))
    uvw, freq = torch.as_tensor(wl.uvw_m).cuda(), torch.as_tensor(wl.freq_hz).cuda()
    pa, sb = torch.as_tensor(wl.pa_bin, dtype=torch.int32).cuda(), torch.as_tensor(wl.chan_subband, dtype=torch.int32).cuda()
    n_plan = _every_failure(hook, lambda: awg.plan_create(cf, uvw, freq, pa, sb))
    assert n_plan >= 10   # records, keys, buckets, scans, items, queues, counters
    # the context still works: a plan, gridding and degridding after all those failures
    plan = awg.plan_create(cf, uvw, freq, pa, sb)
    N = wl.grid_n
    grid = torch.zeros((N, N, 4), dtype=torch.complex64, device="cuda")
    sw = torch.zeros(4, dtype=torch.float64, device="cuda")
    vis = torch.as_tensor(np.asarray(wl.vis).reshape(wl.n_rows, wl.n_chan, 4), dtype=torch.complex64).cuda()
    wt = torch.as_tensor(np.asarray(wl.weight).reshape(wl.n_rows, wl.n_chan, 4), dtype=torch.float32).cuda()
    awg.grid_visibilities(cf, plan, vis, wt, grid, sw)
    out = torch.empty_like(vis)
    awg.degrid_visibilities(cf, plan, grid, out)
    torch.cuda.synchronize()
    assert float(sw.sum()) > 0 and torch.isfinite(torch.view_as_real(out)).all()


def test_cf_set_load_and_autotune_fail_cleanly(hook, tmp_path):
    import paper_2508_17187_gb300 as awg
    wl = synth.make_workload("wproj", n_int=4, n_chan=4, grid_n=512, n_wplanes=4, max_support=24, with_vis=False)
    cf = awg.cf_set_create(**library_params(oracle_params(wl)))
    path = tmp_path / "w.awgcf"
    awg.cf_set_save(cf, path)
    assert _every_failure(hook, lambda: awg.cf_set_load(path)) >= 4
    uvw, freq = torch.as_tensor(wl.uvw_m).cuda(), torch.as_tensor(wl.freq_hz).cuda()

    class _Tuned:   # autotune allocates scratch and plans, and frees all of it on every path
        def __init__(self):
            cf.autotune(uvw, freq, n_pol=4)

        def close(self):
            pass

    assert _every_failure(hook, _Tuned, holds=False) >= 5


def test_hook_rejects_bad_argument(hook):
    assert hook.awg_debug_fail_allocations(-2) == 1
