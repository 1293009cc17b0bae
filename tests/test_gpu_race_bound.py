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


@pytest.mark.parametrize("separable,config", [(True, 0), (False, 0), (True, 2), (True, 3)])
def test_every_pixel_within_its_rounding_bound(separable, config):
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
    if config:   # the warp-specialised kernels on every exact support
        for S in sorted(set(cf.supports().tolist())):
            if S % 8 == 0:
                cf.choose(S, config)
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
    plan.check()
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
    print(f"separable={separable} config={config}: worst pixel at {worst:.3f} of its bound, "
          f"worst sample at {d_worst:.3f}")


def _factor_tables(cf, op, used):
    """FP64 tables of the CFs the kernels evaluate, from their stored FP32 factors: the exact sum
    s * sum_k fy_k fx_k, and |s| * sum_k |fy_k| |fx_k|, which bounds every partial sum of the
    kernels' FP32 evaluation of that sum (tables offset-major [OS+1][OS+1][S][S])."""
    tabs, abst = {}, {}
    for ci in used:
        fx, fy, s = cf.copy_factors(ci)
        fx = fx.astype(np.complex128)
        fy = fy.astype(np.complex128)
        tabs[ci] = complex(s) * np.einsum("kyt,kxs->yxts", fy, fx)
        abst[ci] = abs(complex(s)) * np.einsum("kyt,kxs->yxts", np.abs(fy), np.abs(fx)).astype(np.complex128)
    return tabs, abst


def _check_bounds(g_gpu, g_ref, A, cnt, d_gpu, d_ref, d_abs, taps, slack):
    """Per pixel and per sample: |error| <= (8 + slack + 8 sqrt(n)) u A (slack: the FP32 evaluation
    of each tap's CF value from its terms, and the pol mixing)."""
    bound = (8.0 + slack + 8.0 * np.sqrt(cnt))[:, :, None] * U * A
    err = np.abs(g_gpu - g_ref)
    worst = float((err / np.where(bound > 0, bound, 1.0)).max())
    assert np.all(err <= bound), worst
    assert np.all(g_gpu[A == 0] == 0)
    d_bound = (8.0 + slack + 8.0 * np.sqrt(taps)) * U * d_abs
    d_err = np.abs(d_gpu - d_ref)
    d_worst = float((d_err / np.where(d_bound > 0, d_bound, 1.0)).max())
    assert np.all(d_err <= d_bound), d_worst
    return worst, d_worst


def test_fused_terms_every_pixel_within_its_rounding_bound():
    """The fused kernels of 2-4 CF terms (batched AW-projection, one record per sample, each tap's
    CF value formed from its terms in registers) under the same contention: every pixel and every
    degridded sample within its FP32 rounding bound of the FP64 sum over the stored factors."""
    import paper_2508_17187_gb300 as awg
    from paper_2508_17187_gb300 import _lib
    _lib.load()
    wl = synth.make_workload("awproj", n_int=30, n_chan=8, grid_n=512, n_pa=3, n_sb=2, n_wplanes=8,
                             max_support=64, oversampling=8)
    op = oracle_params(wl)
    N, P = wl.grid_n, wl.n_pol
    n = wl.n_rows * wl.n_chan
    cf = awg.cf_set_create(**library_params(op))
    assert 2 <= cf.fused_terms <= 4
    pa = torch.as_tensor(wl.pa_bin, dtype=torch.int32).cuda()
    sb = torch.as_tensor(wl.chan_subband, dtype=torch.int32).cuda()
    plan = awg.plan_create(cf, torch.as_tensor(wl.uvw_m).cuda(), torch.as_tensor(wl.freq_hz).cuda(), pa, sb)
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

    idx = oindex.sample_index(op, wl.uvw_m, wl.freq_hz, wl.pa_bin, wl.chan_subband)
    used = sorted(set(np.unique(idx.cf[idx.valid]).tolist()))
    tabs, abst = _factor_tables(cf, op, used)
    buf, off, _ = ocf.flatten_cf_set(op, tabs)
    absbuf, _, _ = ocf.flatten_cf_set(op, abst)
    V = wl.vis.reshape(n, P).astype(np.complex128)
    W = wl.weight.reshape(n, P).astype(np.float64)
    OS = op.oversampling
    g_ref, _ = oops.grid(idx, buf, off, OS, N, V, W)
    A, _ = oops.grid(idx, absbuf, off, OS, N, np.abs(V).astype(np.complex128), W)
    cnt, _ = oops.grid(idx, (absbuf.real > 0).astype(np.complex128), off, OS, N, np.ones((n, 1), np.complex128),
                       np.ones((n, 1)))
    A, cnt = A.real, cnt.real[:, :, 0]
    assert cnt.max() > 5000
    d_ref = oops.degrid(idx, buf, off, OS, g_gpu)
    d_abs = oops.degrid(idx, absbuf, off, OS, np.abs(g_gpu).astype(np.complex128)).real
    taps = (idx.support.astype(np.float64) ** 2)[:, None]
    worst, d_worst = _check_bounds(g_gpu, g_ref, A, cnt, d_gpu, d_ref, d_abs, taps, 4.0 * cf.fused_terms)
    print(f"fused {cf.fused_terms} terms: worst pixel at {worst:.3f} of its bound, worst sample at {d_worst:.3f}")


def test_pol_mixing_every_pixel_within_its_rounding_bound():
    """The pol-mixing instances of the fused kernels (full polarisation: three 4-pol passes over the
    base CFs with the Mueller elements' scalars as mixing matrices): every pixel of every pol and
    every degridded sample within its FP32 rounding bound of the FP64 sum over the kept elements."""
    import paper_2508_17187_gb300 as awg
    from paper_2508_17187_gb300 import _lib
    _lib.load()
    wl = synth.make_workload("awproj", n_int=12, n_chan=8, grid_n=512, n_pa=3, n_sb=2, n_wplanes=4,
                             max_support=32, oversampling=8)
    op = oracle_params(wl, use_pol=True, squint_rad=3e-4, leakage=0.04 * np.exp(0.9j), mueller_threshold=0.01)
    N = wl.grid_n
    n = wl.n_rows * wl.n_chan
    cf = awg.cf_set_create(**library_params(op))
    assert cf.fused_terms > 0 and len(cf.mueller()) == 12
    pa = torch.as_tensor(wl.pa_bin, dtype=torch.int32).cuda()
    sb = torch.as_tensor(wl.chan_subband, dtype=torch.int32).cuda()
    plan = awg.plan_create(cf, torch.as_tensor(wl.uvw_m).cuda(), torch.as_tensor(wl.freq_hz).cuda(), pa, sb)
    vis = torch.as_tensor(wl.vis).cuda()
    wt = torch.as_tensor(wl.weight).cuda()
    g = torch.zeros((N, N, 4), dtype=torch.complex64, device="cuda")
    sw = torch.zeros(4, dtype=torch.float64, device="cuda")
    awg.grid_visibilities(cf, plan, vis, wt, g, sw)
    out = torch.empty_like(vis)
    awg.degrid_visibilities(cf, plan, g, out)
    torch.cuda.synchronize()
    g_gpu = g.cpu().numpy().astype(np.complex128)
    d_gpu = out.cpu().numpy().reshape(n, 4).astype(np.complex128)

    idx = oindex.sample_index(op, wl.uvw_m, wl.freq_hz, wl.pa_bin, wl.chan_subband)
    base = sorted(set(np.unique(idx.cf[idx.valid]).tolist()))
    used = [e * op.n_base + c for e in range(len(cf.mueller())) for c in base]
    tabs, abst = _factor_tables(cf, op, used)
    buf, off, _ = ocf.flatten_cf_set(op, tabs)
    absbuf, _, _ = ocf.flatten_cf_set(op, abst)
    V = wl.vis.reshape(n, 4).astype(np.complex128)
    W = wl.weight.reshape(n, 4).astype(np.float64)
    OS = op.oversampling
    g_ref, _ = oops.grid_mueller(op, idx, buf, off, OS, N, V, W)
    A, _ = oops.grid_mueller(op, idx, absbuf, off, OS, N, np.abs(V).astype(np.complex128), W)
    cnt, _ = oops.grid_mueller(op, idx, (absbuf.real > 0).astype(np.complex128), off, OS, N,
                               np.ones((n, 4), np.complex128), np.ones((n, 4)))
    A = A.real
    cnt = cnt.real.max(axis=2)
    assert cnt.max() > 1000
    d_ref = oops.degrid_mueller(op, idx, buf, off, OS, g_gpu)
    d_abs = oops.degrid_mueller(op, idx, absbuf, off, OS, np.abs(g_gpu).astype(np.complex128)).real
    taps = 4.0 * (idx.support.astype(np.float64) ** 2)[:, None]
    worst, d_worst = _check_bounds(g_gpu, g_ref, A, cnt, d_gpu, d_ref, d_abs, taps, 4.0 * cf.fused_terms + 8.0)
    print(f"pol mixing: worst pixel at {worst:.3f} of its bound, worst sample at {d_worst:.3f}")
