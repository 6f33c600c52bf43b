"""The bench's multi-GPU path is replicas: each rank times its own latent and
the job's value uses the slowest rank. Checked here with two gloo ranks on CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = 100.0 if rank == 0 else 250.0   # rank 1 is the slow replica
    total, value = bench.replica_value(local_ms, steps=5, world_size=world, device=torch.device("cpu"))
    q.put((rank, total, value))
    dist.destroy_process_group()


def test_replica_timing_takes_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, total, value in res:
        assert total == 250.0
        assert value == pytest.approx(2 * 5 / 0.25)


def test_single_process_value():
    import bench
    total, value = bench.replica_value(200.0, steps=4, world_size=1, device=torch.device("cpu"))
    assert total == 200.0 and value == pytest.approx(20.0)
