"""The N>1 benchmark path on CPU: two gloo ranks run the same whole-job aggregation the
benchmark uses (slowest rank's time, total pixels over ranks) -- replicas only, no
data-path collective."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms, px = bench.aggregate_ranks(1.0 + rank, 1000 * (rank + 1), world, device="cpu")
        out[rank] = (ms, px)
    finally:
        dist.destroy_process_group()


def test_two_rank_aggregation_gloo():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1] == (2.0, 3000)


def test_single_rank_is_identity():
    import bench
    assert bench.aggregate_ranks(3.5, 123, 1) == (3.5, 123)
