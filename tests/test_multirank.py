"""The multi-GPU (replica) host logic of bench.py on two CPU ranks with the
gloo backend: the whole-job time is the slowest rank's, the points are summed,
every rank gets its own problem, and the reference arm runs on rank 0 only."""

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


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t, p = bench.combine_ranks(1.0 + rank, 100.0 * (rank + 1), world, "cpu")
        seeds = [None] * world
        dist.all_gather_object(seeds, bench.rank_seed(rank))

        class A:  # the reference arm under torchrun: rank 0 alone works
            size = "small"
            steps = 1
            warmup = 0
            gpus = world

        ran = None
        if rank != 0:
            bench.run_reference(A, rank, world)  # returns at once, prints nothing
            ran = False
        dist.barrier()
        q.put((rank, t, p, seeds, ran))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_combine_like_the_benchmark():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    for rank, t, p, seeds, ran in out:
        assert t == 2.0  # max over ranks of 1.0 + rank
        assert p == 300.0  # 100 + 200
        assert len(set(seeds)) == world
        assert ran in (None, False)
