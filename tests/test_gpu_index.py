"""The plan's per-sample index against the oracle, element by element (rows a1 and a2 of the hot
path: the CF_ij(nu, w, t) selection of Eq. CIJ, the pixel and oversampling-offset rules, the drop
rule; readings R4, R6 and R11).

Both sides evaluate the same FP64 steps, each separately rounded, so every integer they derive
must agree exactly: kept / dropped, CF index, first-tap pixel and offsets.  Besides the seeded
W-projection samples, crafted rows at a channel of frequency c (so u_lambda = u_m exactly) put
samples on the plane ties (|w| halfway between two planes), on w = -0, on negative w, on offset
ties (f OS + 1/2 an integer with a dyadic OS) and on both sides of the grid-edge drop limits.
"""
import numpy as np
import pytest

import synth
from oracle import cf as ocf
from oracle import index as oindex
from tests.helpers import library_params, oracle_params

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

C_LIGHT = 299792458.0


@pytest.fixture(scope="module")
def awg():
    import paper_2508_17187_gb300 as m
    from paper_2508_17187_gb300 import _lib
    _lib.load()          # fails loudly when the library is missing: there is no fallback
    assert torch.cuda.is_available()
    return m


def _crafted_rows(op):
    """uvw rows [K, 3] (metres, read at frequency c) hitting the tie and limit cases exactly."""
    N = op.grid_n
    scale = N * op.cell_rad                  # a power of two below: x = u scale + N/2 exactly
    assert scale == 2.0 ** round(np.log2(scale))
    dw = op.w_max_lambda / (op.n_wplanes - 1)
    sup = ocf.supports(op)
    rows = []

    def add(hx, hy, w):
        # the signed plane of w (nearest plane, ties up), its support, then x = hx + S / 2
        k = int(np.floor(abs(w) / dw + 0.5))
        k = min(k, op.n_wplanes - 1)
        ks = op.n_wplanes - 1 + (-k if w < 0 else k)
        S = int(sup[ks])
        x, y = hx + 0.5 * S, hy + 0.5 * S
        rows.append(((x - N // 2) / scale, (y - N // 2) / scale, w))

    OS = op.oversampling
    for k in range(op.n_wplanes + 1):
        for sgn in (1.0, -1.0):
            add(100.0 + k, 140.0, sgn * (k + 0.5) * dw)          # plane tie: goes to the farther plane
            add(120.0, 100.0 + 3 * k, sgn * k * dw)              # exactly on a plane
    add(200.0, 200.0, -0.0)                                      # negative zero: the w >= 0 planes
    for m in range(OS + 1):
        f = (m + 0.5) / OS                                       # offset tie: f OS + 1/2 = m + 1
        add(300.0 - f, 310.0 - (1.0 - f), 0.3 * dw)              # hx = p0x - f with p0x = 300
    add(-1.0, 50.0, 0.0)                                         # on the low limit: kept
    add(-1.0 - 2.0 ** -30, 50.0, 0.0)                            # just below it: dropped
    add(60.0, -1.0, -2.0 * dw)
    add(60.0, -1.0 - 2.0 ** -30, -2.0 * dw)
    for w in (0.0, 3.0 * dw, -(op.n_wplanes - 1) * dw):
        k = min(int(np.floor(abs(w) / dw + 0.5)), op.n_wplanes - 1)
        S = int(sup[op.n_wplanes - 1 + (-k if w < 0 else k)])
        add(N - S - 2.0 ** -30, 70.0, w)                          # just below the high limit: kept
        add(float(N - S), 70.0, w)                                # on it: dropped
        add(80.0, float(N - S), w)
    add(10.0, 10.0, (op.n_wplanes - 0.5) * dw)                   # beyond the last plane: dropped
    add(10.0, 10.0, -(op.n_wplanes - 0.5 + 1e-9) * dw)
    return np.asarray(rows, dtype=np.float64)


@pytest.mark.parametrize("oversampling", [20, 16])
def test_plan_index_equals_oracle_index(awg, oversampling):
    wl = synth.make_workload("wproj", n_int=12, n_chan=4, grid_n=512, n_wplanes=8, max_support=48)
    op = oracle_params(wl, n_wplanes=8, w_max_lambda=7.0 * 65536.0, cell_rad=2.0 ** -20, oversampling=oversampling)
    crafted = _crafted_rows(op)
    uvw = np.concatenate([wl.uvw_m, crafted], 0)
    freq = np.concatenate([[C_LIGHT], wl.freq_hz])
    cf = awg.cf_set_create(**library_params(op))
    plan = awg.plan_create(cf, torch.as_tensor(uvw).cuda(), torch.as_tensor(freq).cuda())
    got = plan.index()
    idx = oindex.sample_index(op, uvw, freq)
    valid = idx.valid
    # the crafted rows exercise what they are meant to: kept and dropped samples, negative w
    R0, C = wl.n_rows, freq.shape[0]
    crafted_valid = valid.reshape(-1, C)[R0:, 0]
    assert crafted_valid.sum() >= 20 and (~crafted_valid).sum() >= 8
    assert (idx.cf[valid] < op.n_wplanes - 1).any() and (idx.cf[valid] > op.n_wplanes - 1).any()
    assert np.array_equal(got["kept"], valid.astype(np.int32))
    for k in ("p0x", "p0y", "ox", "oy"):
        assert np.array_equal(got[k][valid], getattr(idx, k)[valid].astype(np.int32)), k
        assert np.all(got[k][~valid] == -1), k
    assert np.array_equal(got["cf"][valid], idx.cf[valid])
    assert got["ox"][valid].max() <= oversampling and got["ox"][valid].min() >= 0
    st = plan.stats()
    assert st[0] == int(valid.sum()) and st[1] == int((~valid).sum())


def test_plan_index_awproj_bins(awg):
    """PA bins and sub-bands in the CF index (cf = (pa n_sb + sb) n_signed + ks), and a rank-r
    plan (one record per CF term) reports each sample once."""
    wl = synth.make_workload("awproj", n_int=6, n_chan=8, grid_n=512, n_pa=3, n_sb=2, n_wplanes=4, max_support=32)
    op = oracle_params(wl)
    cf = awg.cf_set_create(**library_params(op))
    pa = torch.as_tensor(wl.pa_bin, dtype=torch.int32).cuda()
    sb = torch.as_tensor(wl.chan_subband, dtype=torch.int32).cuda()
    plan = awg.plan_create(cf, torch.as_tensor(wl.uvw_m).cuda(), torch.as_tensor(wl.freq_hz).cuda(), pa, sb)
    got = plan.index()
    idx = oindex.sample_index(op, wl.uvw_m, wl.freq_hz, wl.pa_bin, wl.chan_subband)
    v = idx.valid
    assert np.array_equal(got["kept"], v.astype(np.int32))
    assert np.array_equal(got["cf"][v], idx.cf[v])
    for k in ("p0x", "p0y", "ox", "oy"):
        assert np.array_equal(got[k][v], getattr(idx, k)[v].astype(np.int32)), k
    assert len(np.unique(idx.cf[v] // op.n_signed)) > 3
