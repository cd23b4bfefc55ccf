"""Sharding independent particle sets over ranks (batched and served work):
every set on exactly one rank, loads balanced, and -- run as two gloo ranks
on the CPU -- the per-rank results add up to the single-process result with
no exchange of particle data."""
import os
import socket

import numpy as np
import pytest

from paper_1910_02639_gb300 import workloads as wl
from paper_1910_02639_gb300.batch import shard_sets


def test_every_set_on_exactly_one_rank():
    sizes = [sp[1] for sp in wl.batched_specs(256, seed=1914)]
    for world in (1, 2, 3, 4, 8):
        sh = shard_sets(sizes, world)
        flat = sorted(i for r in sh for i in r)
        assert flat == list(range(len(sizes)))
        loads = [sum(sizes[i] for i in r) for r in sh]
        # greedy largest-first: the spread is at most the largest set
        assert max(loads) - min(loads) <= max(sizes)


def test_shard_edge_cases():
    assert shard_sets([], 3) == [[], [], []]
    assert shard_sets([5], 2) == [[0], []]
    assert shard_sets([3, 3, 3, 3], 2) == [[0, 2], [1, 3]]
    with pytest.raises(ValueError):
        shard_sets([1], 0)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, specs, q):
    import torch
    import torch.distributed as dist
    import oracle
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = shard_sets([sp[1] for sp in specs], world)[rank]
    pairs = 0
    for i in mine:
        s = wl.make_set(*specs[i])
        _, cnt = oracle.OracleTree(s.x, s.y, s.z, bucket_size=16).find(s.h, 64)
        pairs += int(cnt.astype(np.int64).sum())
    t = torch.tensor([pairs, len(mine)], dtype=torch.int64)
    dist.all_reduce(t)  # reporting only, as the benchmark does
    if rank == 0:
        q.put((int(t[0]), int(t[1])))
    dist.destroy_process_group()


def test_two_gloo_ranks_cover_all_sets():
    import multiprocessing as mp
    import oracle
    specs = wl.batched_specs(12, seed=518, nmin=200, nmax=3000)
    ref = 0
    for sp in specs:
        s = wl.make_set(*sp)
        _, cnt = oracle.OracleTree(s.x, s.y, s.z, bucket_size=16).find(s.h, 64)
        ref += int(cnt.astype(np.int64).sum())
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank_main, args=(r, 2, port, specs, q)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in ps)
    pairs, nsets = q.get(timeout=5)
    assert nsets == len(specs) and pairs == ref
