"""The warp-specialised kernels (configuration 2: a producer warp stages chunks into a ring of
shared-memory stages handed over on mbarriers, consumer warps multiply and add; degridding loads
each item's grid window with one TMA tile copy and a reduce warp finishes the sums) and the
tensor-core kernels (configuration 3: each item's window as a 3xTF32 tcgen05 product of operands
built per chunk, accumulated in tensor memory; degridding as a tcgen05 product of the samples' y
factors with TMA-loaded window slices, reduced over x in the epilogue) against
the FP64 oracle on W-projection workloads: every exact support, 1, 2 and 4 pols, the flush modes, a
phase shift, plan reuse across calls, and the bounded waits reporting a withheld hand-over as
AWG_ERR_TIMEOUT.  Gates as in test_gpu_parity (1e-5 relative RMS)."""
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


def _ws_set(awg, op, config=2):
    cf = awg.cf_set_create(**library_params(op))
    sups = sorted(set(cf.supports().tolist()))
    for S in sups:
        assert S % 8 == 0
        cf.choose(S, config)
    return cf, sups


def _oracle(op, wl, grid_for_degrid, phase_shift=None):
    idx = oindex.sample_index(op, wl.uvw_m, wl.freq_hz, phase_shift=phase_shift)
    tabs = ocf.cf_set(op, which=set(np.unique(idx.cf[idx.valid]).tolist()))
    buf, off, _ = ocf.flatten_cf_set(op, tabs)
    n, P = wl.n_rows * wl.n_chan, wl.vis.shape[-1]
    g, sw = oops.grid(idx, buf, off, op.oversampling, op.grid_n, np.asarray(wl.vis).reshape(n, P),
                      np.asarray(wl.weight).reshape(n, P))
    d = oops.degrid(idx, buf, off, op.oversampling, grid_for_degrid.astype(np.complex128))
    return idx, g, sw, d


@pytest.mark.parametrize("config", [2, 3])
@pytest.mark.parametrize("P", [1, 2, 4])
def test_ws_wproj_parity_every_support(awg, P, config):
    wl = synth.make_workload("wproj", n_int=24, n_chan=8, grid_n=1024)
    if P != 4:
        wl.vis = np.ascontiguousarray(wl.vis[..., :P])
        wl.weight = np.ascontiguousarray(wl.weight[..., :P])
    op = oracle_params(wl, n_wplanes=8)
    cf, sups = _ws_set(awg, op, config)
    assert len(sups) >= 6
    N = wl.grid_n
    plan = awg.plan_create(cf, torch.as_tensor(wl.uvw_m).cuda(), torch.as_tensor(wl.freq_hz).cuda())
    vis = torch.as_tensor(wl.vis).cuda()
    wt = torch.as_tensor(wl.weight).cuda()
    g = torch.zeros((N, N, P), dtype=torch.complex64, device="cuda")
    sw = torch.zeros(P, dtype=torch.float64, device="cuda")
    awg.grid_visibilities(cf, plan, vis, wt, g, sw)
    out = torch.full_like(vis, complex(3.0, -1.0))
    awg.degrid_visibilities(cf, plan, g, out)
    plan.check()
    g_np = g.cpu().numpy()
    idx, g_o, sw_o, d_o = _oracle(op, wl, g_np)
    assert rel_rms(g_np, g_o) < 1e-5
    assert np.allclose(sw.cpu().numpy(), sw_o, rtol=1e-12)
    img = oimage.dirty_image(g_np.astype(np.complex128), sw.cpu().numpy(), wl.ps_support)
    img_o = oimage.dirty_image(g_o, sw_o, wl.ps_support)
    assert rel_rms(inner_half(img), inner_half(img_o)) < 1e-5
    d = out.cpu().numpy().reshape(-1, P)
    assert rel_rms(d, d_o) < 1e-5
    for S in sups:   # every support's kernel on its own samples
        m = idx.valid & (idx.support == S)
        if m.any():
            assert rel_rms(d[m], d_o[m]) < 1e-5, S
    assert np.all(d[~idx.valid] == 0)
    # the same plan again: the queues and windows start over
    g2 = torch.zeros_like(g)
    sw2 = torch.zeros_like(sw)
    awg.grid_visibilities(cf, plan, vis, wt, g2, sw2)
    out2 = torch.empty_like(out)
    awg.degrid_visibilities(cf, plan, g, out2)
    plan.check()
    assert rel_rms(g2.cpu().numpy(), g_o) < 1e-5
    assert torch.equal(out2, out)


@pytest.mark.parametrize("config", [2, 3])
@pytest.mark.parametrize("flags", ["kahan", "fp64"])
def test_ws_flush_modes(awg, flags, config):
    wl = synth.make_workload("wproj", n_int=16, n_chan=8, grid_n=512, n_wplanes=6, max_support=40)
    op = oracle_params(wl)
    cf, _ = _ws_set(awg, op, config)
    N, P = wl.grid_n, wl.n_pol
    plan = awg.plan_create(cf, torch.as_tensor(wl.uvw_m).cuda(), torch.as_tensor(wl.freq_hz).cuda())
    sw = torch.zeros(P, dtype=torch.float64, device="cuda")
    if flags == "kahan":
        g = torch.zeros((N, N, P), dtype=torch.complex64, device="cuda")
        glo = torch.zeros_like(g)
        awg.grid_visibilities(cf, plan, torch.as_tensor(wl.vis).cuda(), torch.as_tensor(wl.weight).cuda(), g, sw,
                              grid_lo=glo, flags=awg.AWG_GRID_KAHAN)
        got = g.cpu().numpy().astype(np.complex128) + glo.cpu().numpy().astype(np.complex128)
    else:
        g = torch.zeros((N, N, P), dtype=torch.complex128, device="cuda")
        awg.grid_visibilities(cf, plan, torch.as_tensor(wl.vis).cuda(), torch.as_tensor(wl.weight).cuda(), g, sw,
                              flags=awg.AWG_GRID_FP64)
        got = g.cpu().numpy()
    plan.check()
    _, g_o, sw_o, _ = _oracle(op, wl, np.zeros((N, N, P)))
    # FP32 SIMT kernels: the compensated and FP64 flushes leave the per-item FP32 register sums,
    # well under 1e-6.  Tensor-core gridding: an item's sum runs through the FP32 accumulator of
    # the tensor memory, one rounding per MMA (about 770 over 1024 samples), a few 1e-6 that no
    # flush mode removes; its bound is the FP32 image tolerance.
    assert rel_rms(got, g_o) < (1e-6 if config == 2 else 1e-5)
    assert np.allclose(sw.cpu().numpy(), sw_o, rtol=1e-12)


@pytest.mark.parametrize("config", [2, 3])
def test_ws_phase_shift(awg, config):
    wl = synth.make_workload("wproj", n_int=16, n_chan=8, grid_n=512, n_wplanes=6, max_support=40)
    op = oracle_params(wl)
    cf, _ = _ws_set(awg, op, config)
    N, P = wl.grid_n, wl.n_pol
    shift = (17.0 * wl.cell_rad, -9.0 * wl.cell_rad)
    plan = awg.plan_create(cf, torch.as_tensor(wl.uvw_m).cuda(), torch.as_tensor(wl.freq_hz).cuda(),
                           phase_shift=shift)
    g = torch.zeros((N, N, P), dtype=torch.complex64, device="cuda")
    sw = torch.zeros(P, dtype=torch.float64, device="cuda")
    vis = torch.as_tensor(wl.vis).cuda()
    awg.grid_visibilities(cf, plan, vis, torch.as_tensor(wl.weight).cuda(), g, sw)
    out = torch.empty_like(vis)
    awg.degrid_visibilities(cf, plan, g, out)
    plan.check()
    idx = oindex.sample_index(op, wl.uvw_m, wl.freq_hz, phase_shift=shift)
    tabs = ocf.cf_set(op, which=set(np.unique(idx.cf[idx.valid]).tolist()))
    buf, off, _ = ocf.flatten_cf_set(op, tabs)
    n = wl.n_rows * wl.n_chan
    assert idx.phasor is not None   # the oracle applies it: G by the phasor, D by its conjugate
    g_o, _ = oops.grid(idx, buf, off, op.oversampling, N, wl.vis.reshape(n, P), wl.weight.reshape(n, P))
    d_o = oops.degrid(idx, buf, off, op.oversampling, g.cpu().numpy().astype(np.complex128))
    assert rel_rms(g.cpu().numpy(), g_o) < 1e-5
    assert rel_rms(out.cpu().numpy().reshape(n, P), d_o) < 1e-5


@pytest.mark.parametrize("op_name,config", [("grid", 2), ("degrid", 2), ("grid", 3), ("degrid", 3)])
def test_ws_withheld_handover_times_out_and_context_survives(awg, op_name, config):
    """awg_debug_ws_withhold: the producer of every CTA withholds its first hand-over; the consumers'
    bounded waits give up (2 s), the launch ends, plan_check reports AWG_ERR_TIMEOUT, and the next
    calls on the same context give the oracle's results."""
    from paper_2508_17187_gb300 import _lib
    from paper_2508_17187_gb300._lib import AwgError
    lib = _lib.load()
    wl = synth.make_workload("wproj", n_int=8, n_chan=8, grid_n=512, n_wplanes=4, max_support=8)
    op = oracle_params(wl)
    cf, sups = _ws_set(awg, op, config)
    assert sups == [8]   # one launch per call
    N, P = wl.grid_n, wl.n_pol
    plan = awg.plan_create(cf, torch.as_tensor(wl.uvw_m).cuda(), torch.as_tensor(wl.freq_hz).cuda())
    vis = torch.as_tensor(wl.vis).cuda()
    wt = torch.as_tensor(wl.weight).cuda()
    g = torch.zeros((N, N, P), dtype=torch.complex64, device="cuda")
    sw = torch.zeros(P, dtype=torch.float64, device="cuda")
    out = torch.empty_like(vis)
    assert lib.awg_debug_ws_withhold(1) == 0
    try:
        if op_name == "grid":
            awg.grid_visibilities(cf, plan, vis, wt, g, sw)
        else:
            awg.degrid_visibilities(cf, plan, g, out)
        with pytest.raises(AwgError) as ei:
            plan.check()
        assert ei.value.status == 5   # AWG_ERR_TIMEOUT
    finally:
        lib.awg_debug_ws_withhold(0)
    plan.check()   # the record was cleared
    g.zero_()
    sw.zero_()
    awg.grid_visibilities(cf, plan, vis, wt, g, sw)
    awg.degrid_visibilities(cf, plan, g, out)
    plan.check()
    g_np = g.cpu().numpy()
    _, g_o, sw_o, d_o = _oracle(op, wl, g_np)
    assert rel_rms(g_np, g_o) < 1e-5
    assert rel_rms(out.cpu().numpy().reshape(-1, P), d_o) < 1e-5
