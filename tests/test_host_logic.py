"""Host-side logic that needs no GPU: the DRAM-traffic bookkeeping of bench.py (which sources key
the committed counters, and when they are reported), the partition of work between ranks, and the
marshalling of CF parameters into the C struct."""
import json
import os

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture
def fake_tree(tmp_path, monkeypatch):
    import bench
    csrc = tmp_path / "paper_2508_17187_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "resample_sep.cuh").write_text("// gridding kernels\n")
    (csrc / "clean.cu").write_text("// minor cycle\n")
    (csrc / "notes.txt").write_text("not a source\n")
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "CONFIG", "wproj")
    return bench, csrc, tmp_path


def test_traffic_hash_covers_only_gridding_and_degridding_sources(fake_tree):
    bench, csrc, _ = fake_tree
    h0 = bench.csrc_hash()
    (csrc / "clean.cu").write_text("// minor cycle, changed\n")
    (csrc / "notes.txt").write_text("changed\n")
    assert bench.csrc_hash() == h0           # outside the gridding / degridding launches
    (csrc / "resample_sep.cuh").write_text("// gridding kernels, changed\n")
    assert bench.csrc_hash() != h0
    assert set(bench.NOT_GD_SOURCES) >= {"clean.cu", "gcal.cu", "probe.cu"}


def test_measured_traffic_is_null_unless_current_and_for_this_workload(fake_tree):
    bench, csrc, root = fake_tree
    path = root / "profiles" / "dram_traffic_wproj.json"
    assert bench.measured_traffic("grid") is None                       # no capture committed
    path.write_text(json.dumps({"csrc_sha256": bench.csrc_hash(), "per_launch_bytes": {"grid": 5.0, "degrid": 7.0}}))
    assert bench.measured_traffic("grid") == 5.0 and bench.measured_traffic("degrid") == 7.0
    assert bench.measured_traffic("grid", variant=True) is None         # mosaic / full-pol steps
    (csrc / "resample_sep.cuh").write_text("// kernels changed since the capture\n")
    assert bench.measured_traffic("grid") is None
    path.write_text("{not json")
    assert bench.measured_traffic("grid") is None


@pytest.mark.parametrize("n_parts,world", [(7, 2), (7, 3), (3, 4), (0, 2)])
def test_rank_partitions_cover_every_partition_once(n_parts, world):
    from paper_2508_17187_gb300 import elastic
    got = sorted(p for r in range(world) for p in elastic.owned(n_parts, r, world))
    assert got == list(range(n_parts))


def test_cf_params_marshalling():
    from paper_2508_17187_gb300 import api
    pa = np.array([0.1, -0.2])
    p, keep = api._params(grid_n=512, cell_rad=1e-5, use_a=True, n_pa_bins=2, pa_bin_centers_rad=pa,
                          n_subbands=1, subband_freq_hz=np.array([3e9]), use_pol=True, squint_rad=2e-4,
                          leakage=0.04 * np.exp(0.9j), mueller_threshold=0.01)
    assert (p.grid_n, p.use_a, p.n_pa_bins, p.use_pol) == (512, 1, 2, 1)
    assert p.leakage_re == pytest.approx(0.04 * np.cos(0.9)) and p.leakage_im == pytest.approx(0.04 * np.sin(0.9))
    assert [p.pa_bin_centers_rad[i] for i in range(2)] == [0.1, -0.2]
    assert p.subband_freq_hz[0] == 3e9
    assert len(keep) >= 2   # the arrays the struct points into stay alive with it


def test_bench_rank_slices_tile_the_track():
    """Weak scaling in bench.py: rank r of N takes integrations [r n, (r + 1) n) of a track N n
    long, so the ranks' rows together are the whole track, each row once, with its own PA bins."""
    import bench
    world, n_int = 3, 4
    full = bench.synth.make_workload("wproj", with_vis=False, n_int=world * n_int)
    parts = [bench.rank_workload(world, r, n_int, "cpu", with_vis=False) for r in range(world)]
    assert all(p.n_int == n_int and p.n_rows == n_int * full.n_bl for p in parts)
    assert np.array_equal(np.concatenate([p.uvw_m for p in parts]), full.uvw_m)
    assert np.array_equal(np.concatenate([p.pa_bin for p in parts]), full.pa_bin)
    assert all(p.grid_n == full.grid_n and p.cell_rad == full.cell_rad for p in parts)
