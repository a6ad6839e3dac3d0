"""Replica timing across ranks (bench.py under torchrun) on CPU with gloo,
world size 2: every rank gets the slowest rank's time, and the whole-job rate
counts every replica's units over that time."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = bench.max_over_ranks(1.0 + rank)            # rank 1 is the slow one
    rate = bench.whole_job_rate(1000.0, 4, world, t)
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, t, rate, bench._dist()))


def test_max_over_ranks_gloo_world_2():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, rate, d in res:
        assert t == 2.0
        assert rate == pytest.approx(1000.0 * 4 * 2 / 2.0)
        assert d == (2, rank, rank)


def test_single_process_is_its_own_max():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.whole_job_rate(10.0, 2, 1, 4.0) == 5.0
