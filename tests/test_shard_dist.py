"""Host logic of the replica-sharded path on CPU (no GPU): the shard ranges
cover the solution set, two gloo ranks add their column counts (Eq. 8's sum
over all solutions), agree on Algorithm 2's best solution over the shards
(lowest energy, then the earliest update, then the lowest replica) and
receive the winner's x."""
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
