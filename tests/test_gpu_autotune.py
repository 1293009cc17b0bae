"""The per-support kernel autotuner: it times the four compiled configurations of every
exact-support kernel (two cp.async tilings, the warp-specialised pair, tensor-core gridding) on a plan of the caller's
geometry, keeps the fastest one per support, invalidates older plans, and the tuned set still
matches the oracle."""
import numpy as np
import pytest

import synth
from tests.helpers import library_params, oracle_params, rel_rms

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_autotune_picks_per_support_and_keeps_parity():
    import paper_2508_17187_gb300 as awg
    from paper_2508_17187_gb300._lib import AwgError
    from oracle import cf as ocf
    from oracle import index as oindex
    from oracle import ops as oops
    wl = synth.make_workload("wproj", n_int=24, n_chan=8, grid_n=1024, n_wplanes=8, vis_device="cuda")
    op = oracle_params(wl)
    cf = awg.cf_set_create(**library_params(op))
    uvw = torch.as_tensor(wl.uvw_m).cuda()
    freq = torch.as_tensor(wl.freq_hz).cuda()
    old_plan = awg.plan_create(cf, uvw, freq)
    choice, ms = cf.autotune(uvw, freq, n_pol=4)
    present = set(int(s) for s in np.unique(cf.supports()))
    assert set(choice) == {s for s in present if s % 8 == 0}
    assert all(c in (0, 1, 2, 3) for c in choice.values())
    assert all(min(t) > 0 and len(t) == 4 and ms[s][choice[s]] == min(t) for s, t in ms.items())
    N, P = wl.grid_n, wl.n_pol
    g = torch.zeros((N, N, P), dtype=torch.complex64, device="cuda")
    sw = torch.zeros(P, dtype=torch.float64, device="cuda")
    with pytest.raises(AwgError, match="retuned"):
        awg.grid_visibilities(cf, old_plan, wl.vis, wl.weight, g, sw)
    plan = awg.plan_create(cf, uvw, freq)
    awg.grid_visibilities(cf, plan, wl.vis, wl.weight, g, sw)
    out = torch.empty_like(wl.vis)
    awg.degrid_visibilities(cf, plan, g, out)
    idx = oindex.sample_index(op, wl.uvw_m, wl.freq_hz)
    buf, off, _ = ocf.flatten_cf_set(op, ocf.cf_set(op, which=set(np.unique(idx.cf[idx.valid]).tolist())))
    vis = wl.vis.cpu().numpy().reshape(-1, P).astype(np.complex128)
    wt = wl.weight.cpu().numpy().reshape(-1, P).astype(np.float64)
    g_o, sw_o = oops.grid(idx, buf, off, op.oversampling, N, vis, wt)
    assert rel_rms(g.cpu().numpy(), g_o) < 1e-5
    assert np.allclose(sw.cpu().numpy(), sw_o, rtol=1e-12)
    d_o = oops.degrid(idx, buf, off, op.oversampling, g.cpu().numpy().astype(np.complex128))
    assert rel_rms(out.cpu().numpy().reshape(-1, P), d_o) < 1e-5


def test_choose_rejects_supports_without_configurations():
    import paper_2508_17187_gb300 as awg
    from paper_2508_17187_gb300._lib import AwgError
    wl = synth.make_workload("standard", n_int=4, with_vis=False)
    cf = awg.cf_set_create(**library_params(oracle_params(wl)))
    with pytest.raises(AwgError):
        cf.choose(7, 1)
    with pytest.raises(AwgError):
        cf.choose(8, 4)


def test_autotune_fused_sets_two_configurations_keep_parity():
    """Fused multi-term (AW) sets: the autotuner times configurations 0 and 1 of the fused kernels
    per support, and with configuration 1 on every support gridding and degridding still match the
    FP64 oracle."""
    import paper_2508_17187_gb300 as awg
    from oracle import cf as ocf
    from oracle import index as oindex
    from oracle import ops as oops
    wl = synth.make_workload("awproj", n_int=12, n_chan=8, grid_n=512, n_pa=3, n_sb=2, n_wplanes=4,
                             max_support=32, oversampling=8)
    op = oracle_params(wl)
    cf = awg.cf_set_create(**library_params(op))
    assert cf.fused_terms > 0
    uvw = torch.as_tensor(wl.uvw_m).cuda()
    freq = torch.as_tensor(wl.freq_hz).cuda()
    pa = torch.as_tensor(wl.pa_bin).to(torch.int32).cuda()
    sb = torch.as_tensor(wl.chan_subband).to(torch.int32).cuda()
    choice, ms = cf.autotune(uvw, freq, pa, sb, n_pol=4)
    present = set(int(s) for s in np.unique(cf.supports()))
    assert set(choice) == {s for s in present if s % 8 == 0}
    assert all(c in (0, 1) for c in choice.values())
    assert all(t[0] > 0 and t[1] > 0 and t[2] == 0 and t[3] == 0 for t in ms.values())
    for S in choice:
        cf.choose(S, 1)
    plan = awg.plan_create(cf, uvw, freq, pa, sb)
    N, P = wl.grid_n, wl.n_pol
    vis = torch.as_tensor(wl.vis).cuda()
    wt = torch.as_tensor(wl.weight).cuda()
    g = torch.zeros((N, N, P), dtype=torch.complex64, device="cuda")
    sw = torch.zeros(P, dtype=torch.float64, device="cuda")
    awg.grid_visibilities(cf, plan, vis, wt, g, sw)
    out = torch.empty_like(vis)
    awg.degrid_visibilities(cf, plan, g, out)
    idx = oindex.sample_index(op, wl.uvw_m, wl.freq_hz, wl.pa_bin, wl.chan_subband)
    buf, off, _ = ocf.flatten_cf_set(op, ocf.cf_set(op, which=set(np.unique(idx.cf[idx.valid]).tolist())))
    g_o, sw_o = oops.grid(idx, buf, off, op.oversampling, N, wl.vis.reshape(-1, P).astype(np.complex128),
                          wl.weight.reshape(-1, P).astype(np.float64))
    assert rel_rms(g.cpu().numpy(), g_o) < 1e-5
    assert np.allclose(sw.cpu().numpy(), sw_o, rtol=1e-12)
    d_o = oops.degrid(idx, buf, off, op.oversampling, g.cpu().numpy().astype(np.complex128))
    assert rel_rms(out.cpu().numpy().reshape(-1, P), d_o) < 1e-5
