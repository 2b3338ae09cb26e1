"""One problem over several GPUs: the solution set split into replica shards.

The replicas of IC-D2S interact in two places only: gamma (Eq. 8, a column
sum over all z solutions of the set) and the best solution that Algorithm 2
keeps.  Rank r of a world of W holds the replicas ``shard_range(z, r, W)``
(``icd2s_state_create_shard``: every random draw is keyed by the global
replica index, so the shards together are exactly the set one GPU would
hold).  Per outer iteration a rank runs the Tabu search, adds its column
counts to those of every other rank (one allreduce of n int32) and runs the
rest of the iteration with gamma taken from the totals.  The method's best
solution is the rank best with the smallest (energy, stamp, replica): one
all_gather of three int64 per rank, then a broadcast of the winner's x.

torch.distributed carries the collectives: NCCL on device tensors between
GPUs, or gloo on host tensors (``exchange="cpu"``: the counts are copied to
the host, added and copied back, and the best is chosen on host tensors).
Library calls are enqueued on torch's current stream, which NCCL's
collectives are ordered after; the host copies synchronise with it.
"""
from __future__ import annotations

import numpy as np


def shard_range(z: int, rank: int, world: int) -> tuple[int, int]:
    """(first replica, replica count) of rank `rank`: contiguous, sizes differ by at most one."""
    if not (0 <= rank < world) or z < world:
        raise ValueError("need 0 <= rank < world <= z (z=%d, rank=%d, world=%d)" % (z, rank, world))
    lo, hi = z * rank // world, z * (rank + 1) // world
    return lo, hi - lo


def add_counts(dist, counts, group=None):
    """counts (int32 [n]) <- the sum over every rank's counts, in place."""
    dist.all_reduce(counts, op=dist.ReduceOp.SUM, group=group)
    return counts


def best_owner(dist, torch, mine, device, group=None):
    """mine = (energy, global replica, stamp) of this rank's best (replica -1:
    none yet).  Returns (owner rank, energy, replica, stamp) of the smallest
    (energy, stamp, replica) over the ranks -- Algorithm 2's best: the lowest
    energy, reached first, at the lowest replica of that update."""
    world = dist.get_world_size(group)
    t = torch.tensor([mine[0], mine[2], mine[1]], dtype=torch.int64, device=device)
    allv = [torch.empty_like(t) for _ in range(world)]
    dist.all_gather(allv, t, group=group)
    rows = [tuple(int(v) for v in a.cpu().tolist()) for a in allv]
    cands = [(e, s, r, k) for k, (e, s, r) in enumerate(rows) if r >= 0]
    if not cands:
        return -1, None, -1, -1
    e, s, r, k = min(cands)
    return k, e, r, s


def broadcast_x(dist, torch, x_or_none, n, owner, device, group=None):
    """The owner rank's x (uint8 [n]) on every rank."""
    buf = torch.zeros(n, dtype=torch.uint8, device=device)
    if dist.get_rank(group) == owner:
        buf.copy_(torch.as_tensor(np.ascontiguousarray(x_or_none), dtype=torch.uint8))
    dist.broadcast(buf, src=owner, group=group)
    return buf.cpu().numpy()


class ShardedState:
    """This rank's shard of a solution set of z_total replicas on the current GPU."""

    def __init__(self, I, torch, dist, q, n: int, z_total: int, seed: int, group=None, device="cuda",
                 exchange=None):
        self.I, self.torch, self.dist, self.group, self.device = I, torch, dist, group, device
        self.exchange = exchange or device   # where the collectives' tensors live
        self.n, self.z_total = n, z_total
        rank, world = dist.get_rank(group), dist.get_world_size(group)
        self.base, self.count = shard_range(z_total, rank, world)
        self.st = I.icd2s_state_create_shard(q, self.count, self.base, z_total, seed)
        self.counts = torch.zeros(n, dtype=torch.int32, device=device)

    def close(self):
        if self.st is not None:
            self.I.icd2s_state_destroy(self.st)
            self.st = None

    def _stream(self):
        return self.torch.cuda.current_stream().cuda_stream if self.device == "cuda" else 0

    def initial_pass(self, p):
        """Call_IM_Solution_Set (each replica on its own) and the first best update."""
        s = self._stream()
        self.I.icd2s_initial_pass(self.st, p, s)
        self.I.icd2s_best_update(self.st, s)

    def step(self, p, t: int):
        """Outer iteration t: Tabu, one allreduce of the column counts, the rest."""
        s = self._stream()
        self.I.icd2s_step_shard_begin(self.st, p, t, self.counts.data_ptr(), s)
        if self.exchange == self.device:
            add_counts(self.dist, self.counts, self.group)
        else:
            host = self.counts.to(self.exchange)       # waits for the shard's kernels
            add_counts(self.dist, host, self.group)
            self.counts.copy_(host)
        self.I.icd2s_step_shard_finish(self.st, p, t, self.counts.data_ptr(), s)

    def best(self):
        """(energy, global replica, x) of the method's best over every shard."""
        E, r, stamp = self.I.icd2s_get_best_info(self.st)
        x = self.I.icd2s_get_best(self.st, self.n)[0] if r >= 0 else None
        owner, E, r, _ = best_owner(self.dist, self.torch, (E, r, stamp), self.exchange, self.group)
        if owner < 0:
            return None, -1, None
        return E, r, broadcast_x(self.dist, self.torch, x, self.n, owner, self.exchange, self.group)
