"""The multi-rank host logic on CPU: two gloo ranks shard independent
problems with no overlap and agree on the max-over-ranks time."""

import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1705_02043_gb300 import multi


def test_shard_covers_every_problem_once():
    for nprob in (0, 1, 5, 256, 257):
        for world in (1, 2, 3, 8):
            got = np.concatenate([multi.shard(nprob, r, world) for r in range(world)])
            assert np.array_equal(got, np.arange(nprob))
            sizes = [len(multi.shard(nprob, r, world)) for r in range(world)]
            assert max(sizes) - min(sizes) <= 1


def test_shard_offsets_rebases():
    off = np.array([0, 3, 3, 10, 12, 20])
    rows = []
    for r in range(2):
        a, b, o = multi.shard_offsets(off, r, 2)
        assert o[0] == 0 and o[-1] == b - a
        rows.append((a, b))
    assert rows[0][0] == 0 and rows[0][1] == rows[1][0] and rows[1][1] == 20


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = multi.shard(256, rank, world)
    t = multi.max_over_ranks(1.5 + rank, dist)
    n = multi.sum_over_ranks(len(mine), dist)
    q.put((rank, mine.tolist(), t, n))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=100) for _ in range(2))
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0][2] == res[1][2] == 2.5  # max over ranks
    assert res[0][3] == res[1][3] == 256  # every problem on exactly one rank
    assert not set(res[0][1]) & set(res[1][1])
