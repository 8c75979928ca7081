"""The multi-GPU path of the benchmark is replicas only (one independent
tissue per rank, no data-path collective): the whole-job number is the sum of
the ranks' nodes over the slowest rank's time.  This checks that host logic
with two gloo ranks on the CPU."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r took (r + 1) * 10 ms for its 50 steps of 1024^2 nodes
    ms = bench.max_over_ranks(10.0 * (rank + 1), dist, torch.device("cpu"))
    value = bench.replica_mlups(world, 1024 * 1024, 50, ms * 1e-3)
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, ms, value))


def test_two_replicas_take_the_slowest_rank():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    expect = 2 * 1024 * 1024 * 50 / 0.020 / 1e6
    for rank, ms, value in res:
        assert ms == 20.0
        assert value == pytest.approx(expect)


def test_single_process_needs_no_group():
    import bench
    assert bench.max_over_ranks(3.5, None, None) == 3.5
    assert bench.replica_mlups(1, 1000, 10, 1.0) == pytest.approx(0.01)
