"""The N > 1 path of bench.py on CPU: replicas on two gloo ranks.  Each rank times its own copy of
the workload; the job's time is the slowest rank's and its rate counts the units of all ranks."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = 1000.0 * (rank + 1)  # rank 1 is the slower replica
    worst = bench.max_over_ranks(ms, "cpu")
    dist.barrier()
    q.put((rank, worst, bench.whole_job_rate(4, world, worst)))
    dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_rate_with_two_gloo_ranks():
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
    for rank, worst, rate in got:
        assert worst == 2000.0           # both ranks see the slower replica's time
        assert rate == pytest.approx(4 * 2 / 2.0)  # 8 target-sweeps in 2 s


def test_single_process_is_unchanged():
    import bench
    assert bench.max_over_ranks(123.0, "cpu") == 123.0
    assert bench.whole_job_rate(4, 1, 2000.0) == pytest.approx(2.0)
