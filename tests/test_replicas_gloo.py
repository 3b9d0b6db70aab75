"""The N > 1 path of bench.py on CPU: two gloo ranks, each timing its own
replica; the job time is the slowest rank's and the value counts the updates
of both ranks.  No GPU is involved (the bench runs the same reduction over
NCCL on one GPU per rank)."""
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


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        ms_local = 10.0 + 5.0 * rank          # rank 1 is the slower replica
        ms, value = bench.replica_rate(1.0e9, ms_local, world)
        out[rank] = (ms, value)
    finally:
        dist.destroy_process_group()


def test_two_gloo_replicas_take_the_slowest_rank():
    world = 2
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        got = dict(out)
    for rank in range(world):
        ms, value = got[rank]
        assert ms == 15.0
        assert abs(value - 2.0e9 / 15.0e-3) <= 1e-6 * value


def test_single_rank_needs_no_process_group():
    import bench
    ms, value = bench.replica_rate(3.0e9, 20.0, 1)
    assert ms == 20.0 and abs(value - 1.5e11) < 1.0
