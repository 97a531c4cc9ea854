"""Host logic of the multi-GPU bench (independent replicas, slowest rank
timed) on two gloo ranks on the CPU."""
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


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    local = 1.5 if rank == 0 else 2.5  # each replica's timed seconds
    t = bench.max_over_ranks(local, dist, "cpu")
    out[rank] = (t, bench.aggregate_throughput(512 ** 3, 10, world, t))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_use_slowest_rank():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    assert out[0][0] == 2.5 and out[1][0] == 2.5
    expect = 512 ** 3 * 10 * 2 / 2.5 / 1e6
    assert abs(out[0][1] - expect) < 1e-9 * expect


def test_single_process_is_identity():
    import bench

    assert bench.max_over_ranks(3.0) == 3.0
