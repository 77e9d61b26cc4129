"""Multi-GPU is replicas only: independent systems per rank, the job's step
time is the slowest rank's and simulated time adds over ranks. The host-side
reduction runs here as two gloo ranks on CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = [2.0, 3.0][rank]
    q.put((rank,) + bench.replica_reduce(local_ms, world))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_reduce_two_ranks():
    import multiprocessing as mp
    import bench
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ms, value in out:
        assert ms == 3.0
        assert value == pytest.approx(2 * bench.ns_per_day(3.0))


def test_single_rank_identity():
    import bench
    assert bench.replica_reduce(2.5, 1) == (2.5, bench.ns_per_day(2.5))
