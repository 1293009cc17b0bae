"""Full-size parity on the headline W-projection workload (351 baselines x 2000 integrations x 64
channels x 4 pols, 4096^2 grid, 64 w-planes, OS 20, separable CF storage), with the default kernel
configuration and with the configurations the autotuner picks, which are the ones the bench
times.  The oracle cannot grid 180M visibilities in seconds, so it checks what it can compute on
its own: every sample's keep/drop decision and tap count (bit exact), a band of 16 grid rows
through the dense centre of the uv plane (all samples that touch it), and the degridded values of
20,000 random samples against the oracle's D of the same GPU grid."""
import numpy as np
import pytest

import synth
from oracle import cf as ocf
from oracle import index as oindex
from oracle import ops as oops
from tests.helpers import library_params, oracle_params, rel_rms

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.mark.parametrize("tuned", [False, True], ids=["default", "autotuned"])
def test_wproj_full_size_sampled_parity(tuned):
    import paper_2508_17187_gb300 as awg
    from paper_2508_17187_gb300 import _lib
    _lib.load()
    wl = synth.make_workload("wproj", vis_device="cuda")
    op = oracle_params(wl)
    N, P = wl.grid_n, wl.n_pol
    cf = awg.cf_set_create(**library_params(op))
    assert cf.separable
    uvw = torch.as_tensor(wl.uvw_m).cuda()
    freq = torch.as_tensor(wl.freq_hz).cuda()
    if tuned:
        picks, _ = cf.autotune(uvw, freq, n_pol=P)
        assert 3 in set(picks.values())   # the tensor-core configuration is among those tested
    plan = awg.plan_create(cf, uvw, freq)
    grid = torch.zeros((N, N, P), dtype=torch.complex64, device="cuda")
    sumwt = torch.zeros(P, dtype=torch.float64, device="cuda")
    awg.grid_visibilities(cf, plan, wl.vis, wl.weight, grid, sumwt)
    out = torch.full_like(wl.vis, complex(5.0, 5.0))
    awg.degrid_visibilities(cf, plan, grid, out)
    torch.cuda.synchronize()
    kept, dropped, taps = plan.stats()

    idx = oindex.sample_index(op, wl.uvw_m, wl.freq_hz)
    assert kept == int(idx.valid.sum()) and dropped == int((~idx.valid).sum())
    assert taps == int((idx.support[idx.valid].astype(np.int64) ** 2).sum())

    vis_h = wl.vis.cpu().numpy().reshape(-1, P)
    wt_h = wl.weight.cpu().numpy().reshape(-1, P)
    assert np.allclose(sumwt.cpu().numpy(), wt_h[idx.valid].astype(np.float64).sum(axis=0), rtol=1e-12)

    # band of 16 rows through the centre: every sample whose footprint reaches it
    lo, hi = N // 2 - 8, N // 2 + 8
    touch = idx.valid & (idx.p0y < hi) & (idx.p0y + idx.support > lo)
    sel = np.nonzero(touch)[0]
    sub = oindex.SampleIndex(valid=idx.valid[sel], cf=idx.cf[sel], p0x=idx.p0x[sel], p0y=idx.p0y[sel],
                             ox=idx.ox[sel], oy=idx.oy[sel], support=idx.support[sel])
    used = set(np.unique(idx.cf[idx.valid]).tolist())
    tabs = ocf.cf_set(op, which=used)
    buf, off, _ = ocf.flatten_cf_set(op, tabs)
    band = oops.grid_rows(sub, buf, off, op.oversampling, N, vis_h[sel], wt_h[sel], lo, hi)
    g_band = grid[lo:hi].cpu().numpy()
    assert rel_rms(g_band, band) < 1e-5

    # 20,000 sampled degridded visibilities (dropped ones must be exactly zero)
    rng = np.random.default_rng(5)
    pick = np.sort(rng.choice(idx.valid.size, 20000, replace=False))
    sub2 = oindex.SampleIndex(valid=idx.valid[pick], cf=idx.cf[pick], p0x=idx.p0x[pick], p0y=idx.p0y[pick],
                              ox=idx.ox[pick], oy=idx.oy[pick], support=idx.support[pick])
    g_h = grid.cpu().numpy().astype(np.complex128)
    d_o = oops.degrid(sub2, buf, off, op.oversampling, g_h)
    d = out.cpu().numpy().reshape(-1, P)[pick]
    assert rel_rms(d, d_o) < 1e-5
    assert np.all(d[~sub2.valid] == 0)
