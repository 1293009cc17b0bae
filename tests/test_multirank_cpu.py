"""Multi-rank path on CPU (gloo, world size 2 and 3): every rank grids its own slice of
integrations and one all-reduce sums the planes, which must equal gridding the whole track (the
accumulation over time of Eq. ResIm); the per-rank gridding here is the oracle, the GPU ranks run
the library in its place, with NCCL instead of gloo.  A rank that fails before the collective
(it raises and exits) is detected by the others, whose all-reduce fails; they form a new group and
take over its partitions (paper_2508_17187_gb300.elastic)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, n_int, out_path):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from oracle import cf as ocf
    from oracle import index as oindex
    from oracle import ops as oops
    wl = bench.rank_workload(world, rank, n_int, "cpu")
    op = ocf.CFParams(grid_n=wl.grid_n, cell_rad=wl.cell_rad, oversampling=wl.oversampling, ps_support=7,
                      use_w=True, n_wplanes=wl.n_wplanes, w_max_lambda=wl.w_max_lambda, max_support=wl.max_support)
    idx = oindex.sample_index(op, wl.uvw_m, wl.freq_hz)
    buf, off, _ = ocf.flatten_cf_set(op, ocf.cf_set(op, which=set(np.unique(idx.cf[idx.valid]).tolist())))
    g, sw = oops.grid(idx, buf, off, op.oversampling, op.grid_n, wl.vis.reshape(-1, wl.n_pol),
                      wl.weight.reshape(-1, wl.n_pol), nthreads=2)
    gt = torch.view_as_real(torch.from_numpy(g)).contiguous()
    st = torch.from_numpy(sw)
    dist.all_reduce(gt)
    dist.all_reduce(st)
    if rank == 0:
        np.save(out_path, torch.view_as_complex(gt).numpy())
        np.save(out_path + ".sw.npy", st.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_partition_then_sum_equals_whole(tmp_path, monkeypatch, oracle_built):
    import bench
    from oracle import cf as ocf
    from oracle import index as oindex
    from oracle import ops as oops
    monkeypatch.setitem(__import__("synth").CONFIGS, "wproj",
                        dict(__import__("synth").CONFIGS["wproj"], n_chan=4, grid_n=512, n_wplanes=6, max_support=24))
    world, n_int = 2, 6
    out = str(tmp_path / "grid.npy")
    ctx = mp.get_context("spawn")
    port = _free_port()
    # the child processes see the patched configuration through an environment-free re-patch
    procs = [ctx.Process(target=_patched_rank, args=(r, world, port, n_int, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    # the whole = the ranks' own slices (each rank seeds its own noise) put back together
    import dataclasses
    parts = [bench.rank_workload(world, r, n_int, "cpu") for r in range(world)]
    whole = dataclasses.replace(parts[0], uvw_m=np.concatenate([w.uvw_m for w in parts]),
                                vis=np.concatenate([w.vis for w in parts]),
                                weight=np.concatenate([w.weight for w in parts]))
    op = ocf.CFParams(grid_n=whole.grid_n, cell_rad=whole.cell_rad, oversampling=whole.oversampling, ps_support=7,
                      use_w=True, n_wplanes=whole.n_wplanes, w_max_lambda=whole.w_max_lambda,
                      max_support=whole.max_support)
    idx = oindex.sample_index(op, whole.uvw_m, whole.freq_hz)
    buf, off, _ = ocf.flatten_cf_set(op, ocf.cf_set(op, which=set(np.unique(idx.cf[idx.valid]).tolist())))
    g, sw = oops.grid(idx, buf, off, op.oversampling, op.grid_n, whole.vis.reshape(-1, whole.n_pol),
                      whole.weight.reshape(-1, whole.n_pol))
    got = np.load(out)
    assert np.abs(got - g).max() <= 1e-12 * np.abs(g).max()
    assert np.allclose(np.load(out + ".sw.npy"), sw, rtol=1e-13)


def _patched_rank(rank, world, port, n_int, out):
    import synth
    synth.CONFIGS["wproj"] = dict(synth.CONFIGS["wproj"], n_chan=4, grid_n=512, n_wplanes=6, max_support=24)
    _rank_main(rank, world, port, n_int, out)


def _failover_rank(rank, world, port, n_parts, fail_rank, out_path, when="before"):
    """One rank of the failover test: the partitions' partial sums are small integer tensors (each
    partition p contributes p + 1 in slot p), so the recovered total is checked exactly.  The
    failing rank leaves before the first all-reduce (when="before") or after taking part in the
    first of the two (when="between")."""
    import datetime
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    from paper_2508_17187_gb300 import elastic
    store = dist.TCPStore("127.0.0.1", port, world, rank == 0, timeout=datetime.timedelta(seconds=60))
    dist.init_process_group("gloo", store=store, rank=rank, world_size=world, timeout=datetime.timedelta(seconds=10))

    def compute(parts):
        t = torch.zeros(n_parts, dtype=torch.float64)
        for p in parts:
            t[p] += p + 1
        return [t, torch.tensor([float(len(parts))], dtype=torch.float64)]

    if rank == fail_rank:
        if when == "between":   # its first all-reduce completes everywhere, then it is gone
            dist.all_reduce(compute(elastic.owned(n_parts, rank, world))[0])
        raise SystemExit(3)   # the failure: this rank leaves
    sums, failed = elastic.reduce_with_recovery(compute, n_parts, rank, world, store, timeout_s=10.0, grace_s=2.0)
    np.save(f"{out_path}.{rank}.npy", np.concatenate([sums[0].numpy(), sums[1].numpy(), np.array(failed, float)]))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world,fail_rank,when", [(2, 1, "before"), (3, 2, "before"), (3, 1, "before"),
                                                  (3, 1, "between"), (3, 2, "between")])
def test_rank_failure_is_detected_and_its_partitions_regridded(tmp_path, world, fail_rank, when):
    """A rank that leaves before the all-reduces, or between the first and the second: the others'
    collective fails, the survivors agree on it through the store, form a new group, split the
    failed rank's partitions between them and still sum every partition exactly once (the first
    tensor, already summed with the failed rank's share, is summed again from the kept partials)."""
    n_parts = 7
    port = _free_port()
    out = str(tmp_path / "sums")
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_failover_rank, args=(r, world, port, n_parts, fail_rank, out, when))
             for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    for r, p in enumerate(procs):
        assert p.exitcode == (3 if r == fail_rank else 0), (r, p.exitcode)
    want = np.arange(1, n_parts + 1, dtype=float)
    for r in range(world):
        if r == fail_rank:
            continue
        got = np.load(f"{out}.{r}.npy")
        assert np.array_equal(got[:n_parts], want)        # every partition summed exactly once
        assert got[n_parts] == n_parts                     # partitions gridded over all survivors
        assert list(got[n_parts + 1:]) == [fail_rank]
