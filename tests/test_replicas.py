"""Multi-GPU runs of the benchmark are independent replicas (one process per
GPU, no data-path exchange): the job time is the slowest rank's and the work
is the sum over ranks.  The host-side aggregation is checked here with two
gloo ranks on the CPU."""

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench

        ms, units = bench.reduce_over_ranks(10.0 * (rank + 1), 100 * (rank + 1), "cpu")
        q.put((rank, ms, units))
    finally:
        dist.destroy_process_group()


def test_replica_aggregation_two_ranks():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(world))
    for rank, ms, units in got:
        assert ms == 20.0  # slowest rank
        assert units == 300.0  # 100 + 200


def test_single_process_is_identity():
    import bench

    assert bench.reduce_over_ranks(7.5, 42) == (7.5, 42.0)
