"""Persistent CF cache (cf_set_save / cf_set_load, the on-disk CFCache of Sec. 6): a loaded set holds
the same CF data and kernel choices as the saved one, so its tables and degridded visibilities are
bit for bit those of the original, for every storage mode: separable rank-1 factors, A-term factors
of several terms (fused kernels), a full-polarisation set of base blocks, full FP32 and BF16 tables
and caller tables.  Damaged files are refused."""
import numpy as np
import pytest

import synth
from tests.helpers import library_params, oracle_params

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev(a, dtype=None):
    t = torch.as_tensor(np.asarray(a))
    return (t.to(dtype) if dtype is not None else t).cuda()


def _degrid(awg, cf, wl, P):
    plan = awg.plan_create(cf, _dev(wl.uvw_m), _dev(wl.freq_hz),
                           _dev(wl.pa_bin, torch.int32) if wl.use_a else None,
                           _dev(wl.chan_subband, torch.int32) if wl.use_a else None)
    N = cf.grid_n
    g = torch.Generator(device="cuda").manual_seed(11)
    grid = torch.complex(torch.randn((N, N, P), device="cuda", generator=g),
                         torch.randn((N, N, P), device="cuda", generator=g)).contiguous()
    out = torch.empty((wl.n_rows, wl.n_chan, P), dtype=torch.complex64, device="cuda")
    awg.degrid_visibilities(cf, plan, grid, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _round_trip(awg, tmp_path, cf, wl, P, table_ids):
    path = tmp_path / "set.awgcf"
    awg.cf_set_save(cf, path)
    cf2 = awg.cf_set_load(path)
    assert (cf2.n_cf, cf2.n_values, cf2.rank, cf2.fused_terms) == (cf.n_cf, cf.n_values, cf.rank, cf.fused_terms)
    assert cf2.mueller() == cf.mueller()
    p1, p2 = cf.params(), cf2.params()
    for k in p1:
        assert np.array_equal(np.asarray(p1[k]), np.asarray(p2[k])), k
    for ci in table_ids:
        assert np.array_equal(cf.copy_table(ci), cf2.copy_table(ci)), ci
    assert np.array_equal(_degrid(awg, cf, wl, P), _degrid(awg, cf2, wl, P))
    return path


def test_cf_cache_wprojection_factors_and_kernel_choice(tmp_path):
    import paper_2508_17187_gb300 as awg
    wl = synth.make_workload("wproj", n_int=6, n_chan=8, grid_n=1024, n_wplanes=8, max_support=48, with_vis=False)
    op = oracle_params(wl)
    cf = awg.cf_set_create(**library_params(op))
    cf.choose(16, 1)   # a non-default kernel configuration travels with the file
    _round_trip(awg, tmp_path, cf, wl, 4, [0, op.n_cf // 2, op.n_cf - 1])


def test_cf_cache_aterm_fused_and_full_polarisation(tmp_path):
    import paper_2508_17187_gb300 as awg
    wl = synth.make_workload("awproj", n_int=6, n_chan=8, grid_n=512, n_pa=3, n_sb=2, n_wplanes=4, max_support=32,
                             oversampling=8, with_vis=False)
    op = oracle_params(wl)
    cf = awg.cf_set_create(**library_params(op))
    assert cf.fused_terms > 0
    _round_trip(awg, tmp_path, cf, wl, 4, [0, op.n_cf - 1])
    opp = oracle_params(wl, use_pol=True, squint_rad=3e-4, leakage=0.04 * np.exp(0.9j), mueller_threshold=0.01)
    cfp = awg.cf_set_create(**library_params(opp))
    _round_trip(awg, tmp_path, cfp, wl, 4, [0, opp.n_base + 1, opp.n_cf - 1])


@pytest.mark.parametrize("dtype", [0, 1])
def test_cf_cache_full_tables(tmp_path, dtype):
    import paper_2508_17187_gb300 as awg
    wl = synth.make_workload("standard", n_int=20, with_vis=False)
    op = oracle_params(wl)
    cf = awg.cf_set_create(**library_params(op, cf_dtype=dtype, separable=False))
    assert not cf.separable
    _round_trip(awg, tmp_path, cf, wl, 1, [0])


def test_cf_cache_caller_tables(tmp_path):
    import paper_2508_17187_gb300 as awg
    wl = synth.make_workload("standard", n_int=20, with_vis=False)
    OS, sups = 4, [5, 8, 13]
    rng = np.random.default_rng(3)
    tab = np.concatenate([(rng.standard_normal((OS + 1, OS + 1, S, S)) + 1j * rng.standard_normal((OS + 1, OS + 1, S, S)))
                          .reshape(-1) for S in sups])
    cf = awg.cf_set_create_from_table(sups, tab, grid_n=wl.grid_n, cell_rad=wl.cell_rad, oversampling=OS,
                                      n_pa_bins=len(sups), separable=False, max_support=13)
    path = tmp_path / "tab.awgcf"
    awg.cf_set_save(cf, path)
    cf2 = awg.cf_set_load(path)
    for ci in range(len(sups)):
        assert np.array_equal(cf.copy_table(ci), cf2.copy_table(ci))


def test_cf_cache_refuses_damaged_files(tmp_path):
    import paper_2508_17187_gb300 as awg
    from paper_2508_17187_gb300._lib import AwgError
    wl = synth.make_workload("standard", n_int=10, with_vis=False)
    cf = awg.cf_set_create(**library_params(oracle_params(wl)))
    path = tmp_path / "ok.awgcf"
    awg.cf_set_save(cf, path)
    data = path.read_bytes()
    for cut in (len(data) - 8, len(data) // 2, 200):
        bad = tmp_path / f"cut{cut}.awgcf"
        bad.write_bytes(data[:cut])
        with pytest.raises(AwgError):
            awg.cf_set_load(bad)
    flipped = bytearray(data)
    flipped[-3] ^= 0xff   # the end marker
    bad = tmp_path / "end.awgcf"
    bad.write_bytes(bytes(flipped))
    with pytest.raises(AwgError):
        awg.cf_set_load(bad)
    with pytest.raises(AwgError):
        awg.cf_set_save(cf, tmp_path / "no_such_dir" / "x.awgcf")
    awg.cf_set_load(path)   # the intact file still loads
