"""The multi-GPU mode runs independent replicas: the only cross-rank steps are the
barrier around the timed region and the max over ranks of the elapsed time.  They are
checked here with two CPU processes on the gloo backend."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _rank(rank, world, port, out):
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench.rank_barrier(world)
        mine = 10.0 + 5.0 * rank            # per-rank elapsed ms
        out[rank] = bench.rank_max(mine, world, "cpu")
        bench.rank_barrier(world)
    finally:
        dist.destroy_process_group()


def test_two_replicas_agree_on_the_slowest_rank():
    world, port = 2, _free_port()
    out = mp.get_context("spawn").Manager().dict()
    mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
    assert dict(out) == {0: 15.0, 1: 15.0}


def test_single_process_is_a_no_op():
    import bench
    bench.rank_barrier(1)
    assert bench.rank_max(3.5, 1) == 3.5
