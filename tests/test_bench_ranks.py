"""Multi-rank host logic of bench.py on CPU: two gloo ranks with different step times report the
whole-job throughput over the slowest rank (the path runs one replica per GPU)."""
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


def _rank(rank, world, port, q):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    w, r, lr = bench.dist_env()
    assert (w, r, lr) == (world, rank, rank)
    elapsed = 100.0 + 50.0 * rank  # rank 1 is slower
    value, emax = bench.aggregate_over_ranks(elapsed, agents=1000, steps=10, world=world)
    q.put((rank, value, emax))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_report_whole_job_over_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, value, emax in got:
        assert emax == 150.0
        assert abs(value - 1000 * 10 * 2 / 0.150) < 1e-6


def test_single_rank_is_plain_throughput():
    import bench
    value, emax = bench.aggregate_over_ranks(200.0, agents=500, steps=4, world=1)
    assert emax == 200.0 and abs(value - 500 * 4 / 0.2) < 1e-9
