"""Host logic of bench.py for N > 1 (replicas only): two gloo ranks on CPU.

Each rank runs an independent replica (its own thermal draw, no data-path
collective); the job time is the maximum over ranks and the throughput counts
every rank's atoms."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", init_method="env://", rank=rank, world_size=world)
    wl = bench.make_workload("si_vacancy_215", rank)
    mine = 100.0 + 50.0 * rank
    tmax = bench.max_over_ranks(mine)
    val = bench.job_throughput(wl.system.n, 10, world, tmax)
    q.put((rank, tmax, val, float(wl.system.x[:, :3].sum())))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_max_and_throughput():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    assert all(r[1] == 150.0 for r in res)                   # max over ranks
    assert res[0][2] == pytest.approx(215 * 10 * 2 / 0.150)   # all ranks' atoms
    assert res[0][3] != res[1][3]                            # independent replicas


def test_single_process_defaults():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5) == 12.5
    assert bench.job_throughput(1000, 10, 1, 1000.0) == pytest.approx(1e4)
    a = bench.make_workload("si_vacancy_215", 0)
    b = bench.make_workload("si_vacancy_215", 0)
    assert np.array_equal(a.system.x, b.system.x)
