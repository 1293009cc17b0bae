"""Hogbom minor cycle on the GPU (clean_hogbom) against the FP32 oracle restatement, bit for bit;
its capture in a CUDA graph; and the full major cycle (residual imaging with the library's G and
D, then the minor cycle) on the differentiable-model workload."""
import numpy as np
import pytest

import synth
from tests.helpers import library_params, oracle_params, rel_rms

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dirty(N, n_src, seed, Np=None):
    """A PSF (Np x Np, default 2N) with a main lobe and ringing sidelobes, and a residual made of
    PSF-convolved point sources plus noise (FP32)."""
    rng = np.random.default_rng(seed)
    Np = Np or 2 * N
    yy, xx = np.mgrid[0:Np, 0:Np].astype(np.float64)
    r = np.hypot(yy - Np // 2, xx - Np // 2)
    psf = (np.exp(-r ** 2 / 8.0) + 0.15 * np.cos(r / 2.5) * np.exp(-r / 40.0)).astype(np.float32)
    psf /= psf[Np // 2, Np // 2]
    img = (rng.standard_normal((N, N)) * 0.01).astype(np.float32)
    for _ in range(n_src):
        y, x = rng.integers(N // 8, 7 * N // 8, 2)
        a = np.float32(rng.uniform(0.2, 1.0))
        ya, yb = max(0, y - Np // 2), min(N, y - Np // 2 + Np)
        xa, xb = max(0, x - Np // 2), min(N, x - Np // 2 + Np)
        img[ya:yb, xa:xb] += a * psf[ya - y + Np // 2:yb - y + Np // 2, xa - x + Np // 2:xb - x + Np // 2]
    return psf, img.astype(np.float32)


@pytest.mark.parametrize("N,Np,window", [(256, None, None), (256, None, (64, 192, 40, 200)), (256, None, (3, 250, 5, 200)),
                                         (250, 101, None), (250, 101, (3, 247, 10, 11))])
def test_clean_matches_oracle_bit_for_bit(N, Np, window):
    """N = 256: float4 subtraction and (4-aligned windows) float4 peak search, PSF covering the
    image; an unaligned window takes the scalar search; N = 250 with a 101-pixel PSF: the scalar
    paths and a PSF that overlaps only part of the image (and a one-row window)."""
    import paper_2508_17187_gb300 as awg
    from oracle import clean
    psf, img = _dirty(N, 30, 11, Np)
    res_o, model_o, comps = clean.hogbom(img, psf, 400, 0.1, threshold=0.05, window=window)
    res = torch.as_tensor(img).cuda()
    model = torch.zeros_like(res)
    ws = awg.clean_hogbom(res, model, torch.as_tensor(psf).cuda(), 400, 0.1, 0.05, window)
    assert ws.components() == len(comps)
    assert np.array_equal(model.cpu().numpy(), model_o)
    assert np.array_equal(res.cpu().numpy(), res_o)


def test_clean_replays_from_cuda_graph():
    import paper_2508_17187_gb300 as awg
    N = 256
    psf, img = _dirty(N, 20, 12)
    psf_d = torch.as_tensor(psf).cuda()
    res = torch.as_tensor(img).cuda()
    model = torch.zeros_like(res)
    ws = awg.CleanWorkspace()
    awg.clean_hogbom(res, model, psf_d, 150, 0.2, 0.0, None, ws)
    torch.cuda.synchronize()
    res_e, model_e = res.clone(), model.clone()
    res.copy_(torch.as_tensor(img).cuda())
    model.zero_()
    graph = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        with torch.cuda.graph(graph, stream=side):
            awg.clean_hogbom(res, model, psf_d, 150, 0.2, 0.0, None, ws)
    torch.cuda.current_stream().wait_stream(side)
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(res, res_e) and torch.equal(model, model_e)
    assert ws.components() == 150


def test_major_cycles_with_hogbom_lower_chi2_and_find_sources():
    import paper_2508_17187_gb300 as awg
    from paper_2508_17187_gb300 import autograd as ag
    from paper_2508_17187_gb300 import imaging
    wl = synth.make_workload("autograd", vis_device="cuda")
    op = oracle_params(wl)
    cf = awg.cf_set_create(**library_params(op))
    plan = awg.plan_create(cf, torch.as_tensor(wl.uvw_m).cuda(), torch.as_tensor(wl.freq_hz).cuda())
    fm = ag.ForwardModel(cf, plan, n_pol=1)
    model, hist = imaging.clean_major_cycles(fm, wl.vis, wl.weight, n_major=3, n_minor=300, gain=0.1)
    assert all(b < a for a, b in zip(hist, hist[1:])), hist
    # the search window is the inner half of the field, which holds about 40% of the sources
    assert hist[-1] < 0.8 * hist[0]
    # the brightest components sit on (or next to) true sources inside the search window
    N = wl.grid_n
    sx = np.round(np.asarray(wl.sky_l) / wl.cell_rad).astype(int) + N // 2
    sy = np.round(np.asarray(wl.sky_m) / wl.cell_rad).astype(int) + N // 2
    m = model.cpu().numpy()
    top = np.argsort(-np.abs(m).ravel())[:5]
    for k in top:
        y, x = divmod(int(k), N)
        assert np.min(np.hypot(sy - y, sx - x)) <= 2.0, (y, x)


def test_major_cycle_captured_in_one_graph():
    import paper_2508_17187_gb300 as awg
    from paper_2508_17187_gb300 import autograd as ag
    from paper_2508_17187_gb300 import imaging
    wl = synth.make_workload("autograd", n_int=60, vis_device="cuda")
    op = oracle_params(wl)
    cf = awg.cf_set_create(**library_params(op))
    plan = awg.plan_create(cf, torch.as_tensor(wl.uvw_m).cuda(), torch.as_tensor(wl.freq_hz).cuda())
    fm = ag.ForwardModel(cf, plan, n_pol=1)
    eager = imaging.CleanCycle(fm, wl.vis, wl.weight, n_minor=100)
    eager.step()
    torch.cuda.synchronize()
    cc = imaging.CleanCycle(fm, wl.vis, wl.weight, n_minor=100)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        cc.step()                      # warm-up outside the capture
        cc.model.zero_()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=side):
            cc.step()
    torch.cuda.current_stream().wait_stream(side)
    cc.model.zero_()
    graph.replay()
    torch.cuda.synchronize()
    # the gridding's FP32 atomics make the two residual images differ in the last bits only
    assert rel_rms(cc.model.cpu().numpy(), eager.model.cpu().numpy()) < 1e-2
    assert abs(cc.chi2() - eager.chi2()) <= 1e-4 * eager.chi2()
