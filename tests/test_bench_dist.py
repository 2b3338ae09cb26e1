"""Host logic of bench.py's multi-process path on CPU: two gloo ranks take the
slowest rank's time, the whole-job rate counts every rank's units, and only
rank 0 of the reference arm does work or prints.  No GPU."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = 100.0 + 50.0 * rank             # rank 1 is the slow one
        slowest = bench.max_over_ranks(dist, torch, local_ms, "cpu")
        rate = bench.whole_job_rate(world, 1000, 4, slowest / 1000.0)
        q.put((rank, bench.dist_env(), slowest, rate))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_count_all_units():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=5) for _ in range(world))
    for rank, env, slowest, rate in got:
        assert env == (rank, world, rank)
        assert slowest == 150.0                    # max over ranks, on every rank
        assert rate == pytest.approx(2 * 1000 * 4 / 0.150)


def test_reference_arm_other_ranks_exit_without_output(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class Args:
        steps, warmup, workload = 1, 0, bench.DEFAULT_WORKLOAD
    out = io.StringIO()
    with redirect_stdout(out):
        bench.run_reference(Args(), bench.WORKLOADS[bench.DEFAULT_WORKLOAD])
    assert out.getvalue() == ""
