"""Host logic of bench.py's multi-rank run (independent replicas, no data-path exchange),
on two CPU ranks over gloo: the timing taken is the slowest rank's on every rank, the
whole-job throughput counts every replica, and the reference arm does no work off rank 0."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    own = [0.250, 0.400][rank]  # this rank's elapsed seconds
    t = bench.max_over_ranks(own, dist, "cpu")
    dist.barrier()
    v = bench.replica_mlups(world, 256 ** 3, 100, t)

    class Args:
        steps, warmup, gpus = 5, 3, world

    bench.run_reference(Args, None, rank) if rank != 0 else None  # no work, no output
    out[rank] = (t, v)
    dist.destroy_process_group()


def test_two_gloo_ranks_report_the_slowest_time_and_the_whole_job_throughput():
    world = 2
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    mp.start_processes(_rank, args=(world, _free_port(), out), nprocs=world, join=True,
                       start_method="spawn")
    assert out[0] == out[1]
    t, v = out[0]
    assert t == 0.400
    assert v == pytest.approx(2 * 256 ** 3 * 100 / 0.400 / 1e6)


def test_single_process_uses_its_own_time():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(1.5) == 1.5
    assert bench.replica_mlups(1, 1000, 10, 0.5) == pytest.approx(0.02)
