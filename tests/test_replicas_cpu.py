"""The host side of the multi-GPU bench (replicas only: every rank solves its
own copy, no collective on the data path): the max-over-ranks timing and the
barrier, run as two gloo ranks on the CPU."""

import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, port, q):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=2)
    try:
        import bench

        dist.barrier()
        got = bench.max_over_ranks(1.25 + rank)  # rank 1 is the slower one
        q.put((rank, got))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_with_two_gloo_ranks():
    import multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == {0: 2.25, 1: 2.25}


def test_max_over_ranks_without_a_process_group():
    import bench

    assert bench.max_over_ranks(3.5) == 3.5
