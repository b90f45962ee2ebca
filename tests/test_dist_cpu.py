"""The multi-rank timing rule of bench.py on CPU with gloo, world size 2:
the job's time is the slowest rank's, its throughput every rank's work over
that time.  (On GPUs the path only shards: replicas, no data collective.)"""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [40.0, 55.0][rank]
    gbps, slowest = bench.aggregate(10 ** 9, ms)
    q.put((rank, gbps, slowest, bench.reduce_max(rank + 0.5)))
    dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_aggregate_takes_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = [q.get(timeout=100) for _ in ps]
    for p in ps:
        p.join(timeout=30)
        assert p.exitcode == 0
    for rank, gbps, slowest, mx in out:
        assert slowest == 55.0
        assert abs(gbps - 2e9 / 0.055 / 1e9) < 1e-9
        assert mx == 1.5


def test_single_process_is_identity():
    import bench
    gbps, ms = bench.aggregate(10 ** 9, 50.0)
    assert ms == 50.0 and abs(gbps - 20.0) < 1e-12
