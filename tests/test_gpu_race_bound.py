"""Race check of the gridding and degridding kernels by a per-pixel error bound.

No race detector runs on these GPUs, so the check is numerical.  The FP32 grid is compared pixel
by pixel with the FP64 sum over the same CF values the kernels use (cf_set_copy_table): whatever
the order of the FP32 additions, a pixel of n contributions with absolute sum A = sum |c| w |V|
stays within about sqrt(n) u A of the exact sum (u = 2^-24), so the test allows
(8 + 8 sqrt(n)) u A.  A lost or doubled update (an atomic flush, a shared-window add or a register
accumulator overwritten by another thread) leaves an error of its whole value at that pixel, far
above the bound for all but the smallest CF tail taps.  The workload packs thousands of samples
onto the pixels near the uv origin, so the shared window and the flush atomics run under heavy
contention, over the W-projection supports 8-64, with the separable kernels and with full
tables.  Degridding gets the same per-sample bound, sum over the taps of |c| |grid|.
"""
import numpy as np
import pytest

import synth
from oracle import cf as ocf
from oracle import index as oindex
from oracle import ops as oops
from tests.helpers import library_params, oracle_params

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U = 2.0 ** -24


@pytest.mark.parametrize("separable", [True, False])
def test_every_pixel_within_its_rounding_bound(separable):
    import paper_2508_17187_gb300 as awg
    from paper_2508_17187_gb300 import _lib
    _lib.load()
    wl = synth.make_workload("wproj", n_int=30, n_chan=8, grid_n=512, n_wplanes=8, max_support=64)
    op = oracle_params(wl)
    N, P = wl.grid_n, wl.n_pol
    R, C = wl.n_rows, wl.n_chan
    n = R * C
    cf = awg.cf_set_create(**library_params(op, separable=separable))
    assert cf.separable == separable
    uvw = torch.as_tensor(wl.uvw_m).cuda()
    freq = torch.as_tensor(wl.freq_hz).cuda()
    plan = awg.plan_create(cf, uvw, freq)
    vis = torch.as_tensor(wl.vis).cuda()
    wt = torch.as_tensor(wl.weight).cuda()
    g = torch.zeros((N, N, P), dtype=torch.complex64, device="cuda")
    sw = torch.zeros(P, dtype=torch.float64, device="cuda")
    awg.grid_visibilities(cf, plan, vis, wt, g, sw)
    out = torch.empty_like(vis)
    awg.degrid_visibilities(cf, plan, g, out)
    torch.cuda.synchronize()
    g_gpu = g.cpu().numpy().astype(np.complex128)
    d_gpu = out.cpu().numpy().reshape(n, P).astype(np.complex128)

    idx = oindex.sample_index(op, wl.uvw_m, wl.freq_hz)
    assert idx.valid.all()
    used = sorted(set(np.unique(idx.cf).tolist()))
    tables = {ci: cf.copy_table(ci).astype(np.complex128) for ci in used}
    buf, off, _ = ocf.flatten_cf_set(op, tables)
    absbuf = np.abs(buf).astype(np.complex128)
    V = wl.vis.reshape(n, P).astype(np.complex128)
    W = wl.weight.reshape(n, P).astype(np.float64)
    OS = op.oversampling
    g_ref, _ = oops.grid(idx, buf, off, OS, N, V, W)
    A, _ = oops.grid(idx, absbuf, off, OS, N, np.abs(V).astype(np.complex128), W)
    cnt, _ = oops.grid(idx, (absbuf.real > 0).astype(np.complex128), off, OS, N, np.ones((n, 1), np.complex128),
                       np.ones((n, 1)))
    A, cnt = A.real, cnt.real[:, :, 0]
    assert cnt.max() > 5000                      # heavy contention near the uv origin
    bound = (8.0 + 8.0 * np.sqrt(cnt))[:, :, None] * U * A
    err = np.abs(g_gpu - g_ref)
    worst = float((err / np.where(bound > 0, bound, 1.0)).max())
    assert np.all(err <= bound), worst
    assert np.all(g_gpu[A == 0] == 0)

    d_ref = oops.degrid(idx, buf, off, OS, g_gpu)
    d_abs = oops.degrid(idx, absbuf, off, OS, np.abs(g_gpu).astype(np.complex128)).real
    taps = (idx.support.astype(np.float64) ** 2)[:, None]
    d_bound = (8.0 + 8.0 * np.sqrt(taps)) * U * d_abs
    d_err = np.abs(d_gpu - d_ref)
    d_worst = float((d_err / np.where(d_bound > 0, d_bound, 1.0)).max())
    assert np.all(d_err <= d_bound), d_worst
    print(f"separable={separable}: worst pixel at {worst:.3f} of its bound, worst sample at {d_worst:.3f}")
