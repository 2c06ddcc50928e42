"""The bench's cross-rank figures with two gloo ranks on the CPU: the job's
time is the slowest rank's, its symbols the sum over the ranks (each rank a
replica of the workload), whatever order the ranks finish in."""
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


def _rank(rank, world, port, q):
    import torch
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [120.0, 95.5][rank]
    syms = [400_000_000, 399_999_000][rank]
    got = bench.aggregate_ranks(ms, syms, world, torch.device("cpu"))
    q.put((rank, got))
    dist.barrier()
    dist.destroy_process_group()


def test_aggregate_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in range(2):
        ms, total = res[r]
        assert ms == 120.0
        assert total == 799_999_000.0


def test_aggregate_single_rank():
    import bench
    assert bench.aggregate_ranks(10.0, 123, 1, None) == (10.0, 123.0)
