"""Host logic of the replica-sharded path on CPU (no GPU): the shard ranges
cover the solution set, two gloo ranks add their column counts (Eq. 8's sum
over all solutions), agree on Algorithm 2's best solution over the shards
(lowest energy, then the earliest update, then the lowest replica) and
receive the winner's x; the sharded iteration (with the CUDA library faked)
begins, adds the counts and finishes in that order on every rank."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2502_13947_gb300.shard import shard_range  # noqa: E402


def test_shard_ranges_cover_the_set_in_order():
    for z, world in [(128, 1), (128, 8), (6, 4), (7, 3), (4096, 7)]:
        got = [shard_range(z, r, world) for r in range(world)]
        assert got[0][0] == 0 and sum(c for _, c in got) == z
        for (b0, c0), (b1, _) in zip(got, got[1:]):
            assert b0 + c0 == b1
        assert max(c for _, c in got) - min(c for _, c in got) <= 1
    with pytest.raises(ValueError):
        shard_range(2, 0, 3)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


# per rank: column counts, and (energy, global replica, stamp) of its best
CASES = {
    "lower energy wins": [(-50, 1, 7), (-60, 5, 9)],
    "equal energy: earlier update wins": [(-60, 2, 9), (-60, 4, 4)],
    "equal energy and update: lower replica wins": [(-60, 3, 4), (-60, 4, 4)],
    "a rank with no best yet": [(2 ** 63 - 1, -1, -1), (-1, 6, 1)],
}


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    from paper_2502_13947_gb300 import shard
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        n = 10
        counts = torch.arange(n, dtype=torch.int32) * (rank + 1)
        shard.add_counts(dist, counts)
        out = {"counts": counts.tolist()}
        for name, mine in CASES.items():
            owner, E, r, s = shard.best_owner(dist, torch, mine[rank], "cpu")
            x = np.full(n, rank, np.uint8) if owner == rank else None
            xb = shard.broadcast_x(dist, torch, x, n, owner, "cpu")
            out[name] = (owner, E, r, s, xb.tolist())
        q.put((rank, out))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_add_counts_and_agree_on_the_best():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = dict(q.get(timeout=5) for _ in range(world))
    want_owner = {"lower energy wins": 1, "equal energy: earlier update wins": 1,
                  "equal energy and update: lower replica wins": 0, "a rank with no best yet": 1}
    for rank in range(world):
        assert got[rank]["counts"] == [3 * j for j in range(10)]      # 1x + 2x
        for name, mine in CASES.items():
            owner, E, r, s, xb = got[rank][name]
            assert owner == want_owner[name], name
            assert (E, r, s) == mine[owner]
            assert xb == [owner] * 10                                 # the winner's x everywhere


class _FakeLibrary:
    """Stands in for the CUDA library on CPU: a shard's begin writes counts that
    name its rank, finish records the counts it was handed, so the test sees
    the order of the calls and what crossed the allreduce."""

    def __init__(self, rank, n):
        self.rank, self.n, self.calls = rank, n, []

    def icd2s_state_create_shard(self, q, count, base, total, seed):
        self.calls.append(("create", count, base, total, seed))
        return object()

    def icd2s_state_destroy(self, st):
        self.calls.append(("destroy",))

    def icd2s_initial_pass(self, st, p, s):
        self.calls.append(("initial_pass",))

    def icd2s_best_update(self, st, s):
        self.calls.append(("best_update",))

    def icd2s_step_shard_begin(self, st, p, t, counts_ptr, s):
        import ctypes
        arr = (ctypes.c_int32 * self.n).from_address(counts_ptr)
        for j in range(self.n):
            arr[j] = (self.rank + 1) * (j + t)
        self.calls.append(("begin", t))

    def icd2s_step_shard_finish(self, st, p, t, counts_ptr, s):
        import ctypes
        self.calls.append(("finish", t, list((ctypes.c_int32 * self.n).from_address(counts_ptr))))

    def icd2s_get_best_info(self, st):
        return (-100 + self.rank, 3 * self.rank + 1, 7)      # rank 0's energy is the lowest

    def icd2s_get_best(self, st, n):
        return np.full(n, 10 + self.rank, np.uint8), -100 + self.rank


def _solver_rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    from paper_2502_13947_gb300.shard import ShardedState
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        n = 6
        lib = _FakeLibrary(rank, n)
        sh = ShardedState(lib, torch, dist, None, n, 7, 99, device="cpu")
        sh.initial_pass(None)
        for t in range(3):
            sh.step(None, t)
        E, r, x = sh.best()
        sh.close()
        q.put((rank, lib.calls, E, r, x.tolist()))
    finally:
        dist.destroy_process_group()


def test_sharded_state_orders_its_calls_and_sums_the_counts():
    """The sharded iteration on two gloo ranks with the library faked on CPU:
    each rank creates its shard of the 7 replicas, begins every iteration,
    receives the sum of both ranks' counts before finishing it, and both ranks
    agree on the best solution (rank 0's) and its x."""
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_solver_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = {r: rest for r, *rest in (q.get(timeout=5) for _ in range(world))}
    n = 6
    for rank in range(world):
        calls, E, r, x = got[rank]
        assert calls[0] == ("create", *((3, 0) if rank == 0 else (4, 3)), 7, 99)
        assert calls[1:3] == [("initial_pass",), ("best_update",)]
        for t in range(3):
            assert calls[3 + 2 * t] == ("begin", t)
            assert calls[4 + 2 * t] == ("finish", t, [3 * (j + t) for j in range(n)])   # 1x + 2x
        assert calls[-1] == ("destroy",)
        assert (E, r, x) == (-100, 1, [10] * n)
