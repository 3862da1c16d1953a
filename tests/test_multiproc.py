"""Replica aggregation of bench.py over ranks (gloo, world size 2, CPU).

The solve does not shard: N GPUs run N independent replicas.  The whole-job
rate is the sum of all ranks' DoFs divided by the slowest rank's time."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    dofs = 1000 * (rank + 1)
    t_ms = 10.0 + 5.0 * rank
    rate, tmax = bench.whole_job_rate(dofs, 4, t_ms, world)
    q.put((rank, rate, tmax))
    dist.destroy_process_group()


def test_whole_job_rate_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get() for _ in range(2))
    # (1000 + 2000) DoFs x 4 steps / 15 ms (the slower rank)
    for _, rate, tmax in res:
        assert tmax == 15.0
        assert rate == pytest.approx(3000 * 4 / 0.015)


def test_single_rank_rate():
    sys.path.insert(0, ROOT)
    import bench
    rate, tmax = bench.whole_job_rate(500, 2, 4.0, 1)
    assert rate == pytest.approx(500 * 2 / 0.004) and tmax == 4.0
