"""Replica parallelism: independent energy+gradient evaluations, one process per GPU.

One evaluation of the nested CTMRG does not shard (every column step needs the environment
of the previous one), so several GPUs run independent evaluations -- different seeds, states
of a batch, finite-difference probes -- with no collective on the data path.  The host-side
pieces live here so that they can be tested with ``torch.distributed`` on CPU (gloo):

* ``shard``        which units (evaluations) a rank owns: contiguous, balanced blocks;
* ``timed``        run W warm-up and K timed steps between barriers, return the MAX step
                   time over ranks (the whole job is as slow as its slowest rank);
* ``max_over_ranks`` the maximum of a per-rank number (what ``bench.py`` reports);
* ``gather``       collect per-rank results on every rank, in unit order.
"""
from __future__ import annotations

import time
from typing import Any, Callable, List, Sequence


def _dist():
    import torch.distributed as dist
    return dist if dist.is_available() and dist.is_initialized() else None


def shard(n_units: int, rank: int, world: int) -> range:
    """Units [lo, hi) of this rank; sizes differ by at most one, lower ranks take the extra."""
    if world < 1 or not 0 <= rank < world or n_units < 0:
        raise ValueError("bad shard arguments")
    base, extra = divmod(n_units, world)
    lo = rank * base + min(rank, extra)
    return range(lo, lo + base + (1 if rank < extra else 0))


def timed(step: Callable[[], None], steps: int, warmup: int, sync: Callable[[], None] = lambda: None,
          clock: Callable[[], float] = time.perf_counter) -> float:
    """Seconds for ``steps`` calls of ``step`` after ``warmup`` untimed ones, max over ranks.

    ``sync`` waits for the device (e.g. ``torch.cuda.synchronize``); it runs together with a
    barrier on both sides of the timed region.
    """
    dist = _dist()
    for _ in range(warmup):
        step()
    sync()
    if dist:
        dist.barrier()
    t0 = clock()
    for _ in range(steps):
        step()
    sync()
    dt = clock() - t0
    if dist:
        dist.barrier()
    return max_over_ranks(dt)


def max_over_ranks(x: float) -> float:
    """The largest value of x over all ranks (x itself without a process group)."""
    import torch

    dist = _dist()
    if not dist:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64)
    if dist.get_backend() == "nccl":
        t = t.cuda()
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t[0])


def gather(local: Sequence[Any], n_units: int) -> List[Any]:
    """Per-unit results of every rank, in unit order, on every rank (host objects)."""
    dist = _dist()
    if not dist:
        return list(local)
    world = dist.get_world_size()
    parts: List[Any] = [None] * world
    dist.all_gather_object(parts, list(local))
    out: List[Any] = []
    for r in range(world):
        rng = shard(n_units, r, world)
        if len(parts[r]) != len(rng):
            raise RuntimeError(f"rank {r} returned {len(parts[r])} results for {len(rng)} units")
        out.extend(parts[r])
    return out
