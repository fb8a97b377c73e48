"""The benchmark's cross-rank aggregation with two gloo ranks on the CPU: whole-job
throughput is the sum of the ranks' pairs over the slowest rank's time."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r processed (r+1) * 1e9 pairs in (r+1) * 100 ms
    value, ms = bench.aggregate((rank + 1) * 1e9, (rank + 1) * 100.0, device="cpu")
    out[rank] = (value, ms)
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_aggregate_two_gloo_ranks(world):
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    # total 3e9 pairs over the slowest rank's 200 ms = 15 G pairs/s, seen by every rank
    for r in range(world):
        value, ms = res[r]
        assert ms == 200.0
        assert abs(value - 15.0) < 1e-9


def test_aggregate_single_process():
    import bench
    value, ms = bench.aggregate(2e9, 400.0)
    assert ms == 400.0 and abs(value - 5.0) < 1e-12
