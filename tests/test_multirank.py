"""The replicas-over-ranks bookkeeping of bench.py on CPU with two gloo
ranks: each rank times its own work, the job's time is the slowest rank's
(max over ranks) and the whole-job rate counts every rank's units."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, lr = bench.rank_env()
    t = 1.0 + rank  # rank 1 is the slow one
    tmax = bench.max_over_ranks(t)
    dist.barrier()
    out.put((r, w, lr, tmax, bench.job_rate(w, 1000, tmax)))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    assert [r[0] for r in res] == [0, 1]
    for r, w, lr, tmax, rate in res:
        assert w == 2 and lr == r
        assert tmax == 2.0  # the slowest rank's time, on every rank
        assert rate == 2 * 1000 / 2.0


def test_single_process_is_its_own_max():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.job_rate(1, 10, 2.0) == 5.0
