"""Multi-process (N > 1) path of bench.py on CPU with the gloo backend.

The traversal does not shard (a distributed BFS would exchange the
frontier every round), so N GPUs run N independent replicas; the only
collective is the max-over-ranks of the elapsed time.  World size 2."""
import os
import socket

import pytest


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
    local_ms = [120.0, 200.0][rank]
    value, tmax = bench.replica_throughput(local_ms, world, units_per_step=1000, steps=5, dist=dist)
    q.put((rank, value, tmax))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_throughput_gloo_world2():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, value, tmax in res:
        assert tmax == 200.0                     # slowest rank decides
        assert value == pytest.approx(2 * 1000 * 5 / 200.0)


def test_replica_throughput_single():
    import bench
    v, t = bench.replica_throughput(50.0, 1, 10, 4)
    assert t == 50.0 and v == pytest.approx(0.8)
