"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): the step
time is the max over ranks and the throughput aggregates every rank's
(independent, weak-scaled) field."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = bench.max_over_ranks(10.0 + 5.0 * rank)  # rank 1 is the slow one
    val = bench.job_throughput(bench.UNKNOWNS_PER_STEP, world, ms)
    q.put((rank, ms, val))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_gloo():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, ms, val in out:
        assert ms == 15.0
        assert val == pytest.approx(2 * 3 * 512 ** 3 / 15e-3 / 1e9)


def test_single_process_identity():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.job_throughput(1e9, 1, 1000.0) == pytest.approx(1.0)
