"""Multi-rank host logic on CPU: two gloo ranks shard a quartet list with no
data exchange and reduce their step times by maximum."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2605_10312_gb300 import shard, synth


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, result):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    _, q = synth.class_sweep((1, 1, 0, 0), 101, seed=4)
    mine = shard.shard_quartets(q, rank, world)
    t = shard.max_over_ranks(10.0 + rank)
    n = shard.sum_over_ranks(mine.shape[0])
    result[rank] = (mine.tolist(), t, n)
    dist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        result = m.dict()
        procs = [ctx.Process(target=_rank_main, args=(r, world, port, result)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(result)
    _, q = synth.class_sweep((1, 1, 0, 0), 101, seed=4)
    got = [tuple(x) for r in range(world) for x in res[r][0]]
    assert sorted(got) == sorted(tuple(x) for x in q.tolist())
    assert [len(res[r][0]) for r in range(world)] == shard.shard_sizes(q.shape[0], world)
    assert all(res[r][1] == 11.0 for r in range(world))
    assert all(res[r][2] == q.shape[0] for r in range(world))


def test_shard_errors():
    q = np.zeros((5, 4), np.int32)
    with pytest.raises(ValueError):
        shard.shard_quartets(q, 2, 2)
    assert shard.shard_sizes(5, 3) == [2, 2, 1]
    assert shard.max_over_ranks(3.5) == 3.5
