"""Multi-GPU is replicas only (fields are independent): each rank times its own batch
and the job's throughput is all ranks' fields over the slowest rank's time. The
aggregation runs here on CPU with two gloo ranks."""
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms, fields = bench.aggregate(100.0 + 50.0 * rank, 64 * 10, world)
        out[rank] = (ms, fields)
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_replica_aggregation_gloo(world):
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert len(res) == world
    for r in range(world):
        assert res[r] == (150.0, 64.0 * 10 * world)    # slowest rank's time, all ranks' fields


def test_single_process_aggregation_is_identity():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate(12.5, 640, 1) == (12.5, 640.0)
