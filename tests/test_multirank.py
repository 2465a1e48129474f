"""N > 1 path of bench.py on CPU: independent replicas (one shot per rank),
no data-path collective; the timing is the max over ranks and the value is
all ranks' units over that time.  world_size 2, gloo, 127.0.0.1."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [120.0, 180.0][rank]
    out = bench.aggregate(ms, 1000.0, dist, torch.device("cpu"))
    q.put((rank, out))
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_aggregate_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(2):
        ms, rate = res[r]
        assert ms == pytest.approx(180.0)
        assert rate == pytest.approx(2 * 1000.0 / 0.18)


def test_single_process_aggregate():
    import bench
    ms, rate = bench.aggregate(250.0, 500.0)
    assert ms == 250.0 and rate == pytest.approx(2000.0)
