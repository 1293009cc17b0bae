"""Multi-rank path on CPU (gloo, world size 2): every rank grids its own slice of integrations and
one all-reduce sums the planes, which must equal gridding the whole track (the accumulation over
time of Eq. ResIm).  The per-rank gridding here is the oracle; the GPU ranks run the library in
its place, with NCCL instead of gloo."""
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
