"""The bench's multi-process path on CPU: two gloo ranks each run their own replica (no data-path collective)
and the reported time is the maximum over ranks, the value the sum of all ranks' work divided by it."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench.barrier(dist)
        t = bench.max_over_ranks(dist, 1.0 + rank)            # per-rank "time"
        g = bench.sum_over_ranks(dist, 100.0 * (rank + 1))    # per-rank "gates"
        out[rank] = (t, g)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_max_and_sum_over_two_gloo_ranks(world):
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        t, g = res[r]
        assert t == 2.0          # max over ranks of 1.0, 2.0
        assert g == 300.0        # 100 + 200


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(None, 3.5) == 3.5
    assert bench.sum_over_ranks(None, 7.0) == 7.0
