"""Multi-rank host logic on CPU with the gloo backend (world size 2): instance
sharding and the max-over-ranks timing, no GPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2509_13592_gb300 import shard


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_partition_balances_cost_and_covers_every_instance():
    shapes = [(64, 64), (256, 256), (128, 64), (256, 128), (64, 256), (128, 128), (256, 256), (64, 64)] * 5
    parts = shard.partition(shapes, 3)
    flat = sorted(i for p in parts for i in p)
    assert flat == list(range(len(shapes)))
    loads = [sum(shard.instance_cost(*shapes[i]) for i in p) for p in parts]
    assert max(loads) - min(loads) <= max(shard.instance_cost(*s) for s in shapes)
    assert shard.partition(shapes, 1) == [list(range(len(shapes)))]
    with pytest.raises(ValueError):
        shard.partition(shapes, 0)


def _worker(rank, world, port, out):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = list(shard.contiguous_range(4, rank))
        elapsed = 1.5 + rank  # a stand-in for each rank's timed region
        out[rank] = (mine, shard.max_over_ranks(elapsed))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_take_the_max():
    port = _free_port()
    # spawn, not fork: earlier tests may have left threads (BLAS, FFT workers) in this process
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0][0] == [0, 1, 2, 3] and res[1][0] == [4, 5, 6, 7]
    assert res[0][1] == res[1][1] == 2.5
    assert shard.max_over_ranks(7.0) == 7.0  # no process group: identity
