"""Weak scaling over time slices with rank-failure recovery (the HTC parallelism of Sec. 4.1.1 as
one process per GPU on a node).  Every rank grids its own partitions of the integrations; one
all-reduce sums the planes (the accumulation over t of Eq. ResIm).  When a rank fails - raises,
exits, or never reaches the collective - the all-reduce of the others ends with an error (a peer
that closed its connection, or the process group's timeout).  The survivors then announce
themselves in the job's store, form a new process group among themselves, take over the failed
ranks' partitions (split round-robin) and sum again.

Host-side coordination only: nothing here runs on or waits in a GPU kernel.  Rank 0 hosts the
store, so its own failure ends the job.  A survivor must reach the recovery within `grace_s`
seconds of the first one (it does: the failed collective returns to every survivor at once).
"""
from __future__ import annotations

import datetime
import time
from typing import Callable, List, Sequence, Tuple

import torch
import torch.distributed as dist


def owned(n_parts: int, rank: int, world: int) -> List[int]:
    """The partitions rank `rank` of `world` grids first: p = rank, rank + world, ..."""
    return list(range(rank, n_parts, world))


_calls = [0]   # reduce_with_recovery calls made by this process (every rank makes them in the same order)


def _agree(store, key: str, rank: int, world: int, mine: str, wait_s: float) -> dict:
    """Publish this rank's outcome under key/<rank>, then collect every rank's outcome, waiting at
    most wait_s for the missing ones; a rank that never publishes (it died) is absent."""
    rank_key = f"{key}/{{}}"
    store.set(rank_key.format(rank), mine)
    deadline = time.monotonic() + wait_s
    seen = {}
    while True:
        for r in range(world):
            if r not in seen and store.check([rank_key.format(r)]):
                seen[r] = store.get(rank_key.format(r)).decode()
        if len(seen) == world or time.monotonic() >= deadline:
            return seen
        time.sleep(0.05)


def reduce_with_recovery(compute: Callable[[Sequence[int]], List[torch.Tensor]], n_parts: int, rank: int, world: int,
                         store, backend: str = "gloo", timeout_s: float = 10.0,
                         grace_s: float = 2.0) -> Tuple[List[torch.Tensor], List[int]]:
    """Sum over all n_parts partitions of the tensors compute(parts) returns (partial sums of the
    given partitions, the same shapes for any list, zeros for an empty one), across the ranks of the
    default process group, which must have been initialised with `store`.  Returns (the sums, the
    ranks that failed).  After a failure the default process group is the survivors' group (ranks
    renumbered in order).

    The ranks agree on the outcome through the store before returning: every rank publishes whether
    all of its all-reduces completed, and the sums are returned only when every rank of the world
    published success.  Otherwise - a collective failed on some rank, or a rank never published
    (it died, possibly between two all-reduces, after some ranks had completed the first) - every
    survivor discards what the all-reduces left and sums again from its own partial sums."""
    call = _calls[0]
    _calls[0] += 1
    partial = compute(owned(n_parts, rank, world))
    keep = [t.clone() for t in partial]   # an interrupted all-reduce may leave a tensor half summed
    ok = True
    try:
        for t in partial:
            dist.all_reduce(t)
    except RuntimeError:
        ok = False
    outcomes = _agree(store, f"elastic/{call}/outcome", rank, world, "ok" if ok else "fail", timeout_s + grace_s)
    if len(outcomes) == world and all(v == "ok" for v in outcomes.values()):
        return partial, []
    # recovery: the survivors are the ranks that published an outcome
    survivors = sorted(outcomes)
    failed = [r for r in range(world) if r not in survivors]
    new_rank, new_world = survivors.index(rank), len(survivors)
    dist.destroy_process_group()
    dist.init_process_group(backend, store=dist.PrefixStore(f"elastic/{call}/recovery", store), rank=new_rank,
                            world_size=new_world, timeout=datetime.timedelta(seconds=timeout_s))
    lost = [p for r in failed for p in owned(n_parts, r, world)]
    extra = compute(lost[new_rank::new_world])
    for k, t in zip(keep, extra):
        k += t
    for t in keep:
        dist.all_reduce(t)
    return keep, failed
