"""Replica parallelism on CPU: shard / timed / gather with two gloo ranks (no GPU needed)."""
import json
import os
import socket
import time

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import workloads as W
from paper_2512_14414_gb300.replicas import gather, max_over_ranks, shard, timed


@pytest.mark.parametrize("world", [1, 2, 3, 4])
def test_shard_partitions_the_units(world):
    for n in range(0, 11):
        parts = [list(shard(n, r, world)) for r in range(world)]
        assert sum(parts, []) == list(range(n))
        sizes = [len(p) for p in parts]
        assert max(sizes) - min(sizes) <= 1


def _energies(seeds):
    # one unit = one oracle evaluation of a small PEPS (D=2, chi=4, 2 iterations)
    from oracle.api import evaluate
    out = []
    for s in seeds:
        w = W.custom(1, 1, 2, 4, 2, seeds=[s], terms=W.heisenberg_terms_rotated())
        E, _ = evaluate(w.tensors, w.Lx, w.Ly, w.chi, w.n_iter, w.terms, env0=W.initial_environment(w), grad=False)
        out.append(float(E))
    return out


def _rank_main(rank, world, port, outdir, seeds):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = [seeds[i] for i in shard(len(seeds), rank, world)]
        got = gather(_energies(mine), len(seeds))
        dt = timed(lambda: time.sleep(0.02 * (rank + 1)), steps=3, warmup=1)
        mx = max_over_ranks(float(rank + 7))
        with open(os.path.join(outdir, f"rank{rank}.json"), "w") as f:
            json.dump({"energies": got, "dt": dt, "max": mx}, f)
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_gather_in_unit_order_and_time_the_slowest(tmp_path):
    seeds = [0, 1, 2, 3, 4]
    mp.start_processes(_rank_main, args=(2, _free_port(), str(tmp_path), seeds), nprocs=2, join=True,
                       start_method="spawn")
    serial = _energies(seeds)
    for r in range(2):
        d = json.load(open(tmp_path / f"rank{r}.json"))
        assert np.allclose(d["energies"], serial, rtol=0, atol=1e-14)
        # the slower rank sleeps 3 x 0.04 s: every rank reports at least that
        assert d["dt"] >= 0.12 - 1e-3
        assert d["max"] == 8.0
