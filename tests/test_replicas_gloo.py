"""The multi-GPU path is replicas only (independent molecules, no exchange): the host-side
aggregation of bench.py (barrier, max over ranks, whole-job atoms/s) with 2 gloo ranks on
the CPU."""
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


def _rank(rank, ws, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    dist.barrier()
    # rank r took 1 + r seconds for 20 steps of 5,000 atoms
    v = bench.replica_throughput(1.0 + rank, ws, 5000, 20, "cpu")
    out[rank] = v
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    ws, port = 2, _free_port()
    out = mp.get_context("spawn").Manager().dict()
    mp.spawn(_rank, args=(ws, port, out), nprocs=ws, join=True)
    expect = ws * 5000 * 20 / 2.0
    assert out[0] == pytest.approx(expect) and out[1] == pytest.approx(expect)


def test_one_replica_needs_no_process_group():
    import bench
    assert bench.replica_throughput(0.5, 1, 1000, 10) == pytest.approx(20000.0)
