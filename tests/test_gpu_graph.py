"""The hot path inside one captured CUDA graph: plan update, gridding, normalisation and
degridding are stream-ordered device work with no host synchronisation or allocation, so a step
captured once replays with the results of the eager calls (degridding bit for bit; gridding up to
the order of its FP32 atomic flushes)."""
import numpy as np
import pytest

import synth
from tests.helpers import library_params, oracle_params, rel_rms

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("config", ["wproj", "awproj", "wproj_ws", "wproj_mma"])
def test_step_replays_from_cuda_graph(config):
    import paper_2508_17187_gb300 as awg
    if config in ("wproj", "wproj_ws", "wproj_mma"):
        wl = synth.make_workload("wproj", n_int=24, n_chan=8, grid_n=1024, n_wplanes=8, vis_device="cuda")
    else:
        wl = synth.make_workload("awproj", n_int=12, n_chan=8, grid_n=512, n_pa=3, n_sb=2, n_wplanes=4,
                                 max_support=32, oversampling=8, vis_device="cuda")
    op = oracle_params(wl)
    cf = awg.cf_set_create(**library_params(op))
    if config in ("wproj_ws", "wproj_mma"):   # warp-specialised / tensor-core kernels (tensor maps built at capture)
        for S in sorted(set(cf.supports().tolist())):
            cf.choose(S, 2 if config == "wproj_ws" else 3)
    uvw = torch.as_tensor(wl.uvw_m).cuda()
    freq = torch.as_tensor(wl.freq_hz).cuda()
    pa = torch.as_tensor(wl.pa_bin).cuda() if wl.use_a else None
    sb = torch.as_tensor(wl.chan_subband).cuda() if wl.use_a else None
    plan = awg.plan_create(cf, uvw, freq, pa, sb)
    N, P = wl.grid_n, wl.n_pol
    rng = np.random.default_rng(5)
    model = torch.as_tensor((rng.standard_normal((N, N, P)) + 1j * rng.standard_normal((N, N, P))).astype(np.complex64)).cuda()
    grid = torch.zeros((N, N, P), dtype=torch.complex64, device="cuda")
    sumwt = torch.zeros(P, dtype=torch.float64, device="cuda")
    out = torch.empty_like(wl.vis)

    def step():
        plan.update(uvw, freq, pa, sb)
        grid.zero_()
        sumwt.zero_()
        awg.grid_visibilities(cf, plan, wl.vis, wl.weight, grid, sumwt)
        awg.grid_normalize(cf, grid, sumwt, direction=0)
        awg.degrid_visibilities(cf, plan, model, out)

    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        for _ in range(2):
            step()
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    g_eager, w_eager, o_eager = grid.clone(), sumwt.clone(), out.clone()

    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step()
    grid.fill_(7.0)
    out.fill_(-3.0)
    for _ in range(2):
        graph.replay()
        torch.cuda.synchronize()
        assert torch.equal(out, o_eager)
        assert torch.allclose(sumwt, w_eager, rtol=1e-12, atol=0)
        assert rel_rms(grid.cpu().numpy(), g_eager.cpu().numpy()) < 1e-6
