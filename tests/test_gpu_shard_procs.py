"""GPU: the replica-sharded path through torch.distributed with real ranks.
Two processes share the one GPU, each holding a shard of the solution set;
they add their column counts (Eq. 8) with a gloo allreduce of host tensors
between the two halves of every outer iteration and choose Algorithm 2's
best over the shards.  The concatenated shards equal the whole set run on
one state in this process, and the oracle's run.  No kernel of one rank
waits on the other rank: every exchange happens on the host between
launches."""
import datetime
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2502_13947_gb300 import build as B
from paper_2502_13947_gb300 import icd2s as I
from paper_2502_13947_gb300.instances import make_qubo

from .gpu_util import lib_params, orc_params, torch_cuda

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    torch_cuda()
    B.build()
    return I.lib()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, Q, kw, seed, iters, out):
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    from paper_2502_13947_gb300 import icd2s as I
    from paper_2502_13947_gb300.shard import ShardedState
    torch.cuda.set_device(0)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=120))
    n = Q.shape[0]
    q = I.icd2s_qubo_create(Q)
    p = I.icd2s_default_params(n)
    for k, v in kw.items():
        setattr(p, k, v)
    sh = ShardedState(I, torch, dist, q, n, z_total=kw["z"], seed=seed, device="cuda", exchange="cpu")
    try:
        sh.initial_pass(p)
        per_iter = []
        for t in range(iters):
            sh.step(p, t)
            x, _, E = I.icd2s_get_state(sh.st, sh.count, n)
            per_iter.append((x, E))
        E, r, bx = sh.best()
        out.put((rank, sh.base, per_iter, (E, r, None if bx is None else np.asarray(bx))))
    finally:
        sh.close()
        I.icd2s_qubo_destroy(q)
        dist.destroy_process_group()


@pytest.mark.parametrize("case", ["plain", "uneven batch"])
def test_two_ranks_on_one_gpu_evolve_like_the_whole_set_and_the_oracle(L, orc, case):
    torch = torch_cuda()
    n, iters, seed, world = 300, 4, 23, 2
    Q = make_qubo(n, 0.5, 19)
    kw = dict(z=6, K=1, m_min=24, m_max=24, m_init=24, alpha=n, c=3, sweeps=24, T_max=1500.0, mut_mode=0,
              patience=0, max_iters=iters)
    if case == "uneven batch":
        kw.update(K=4, m_min=8, m_max=40, m_init=32)
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, Q, kw, seed, iters, out)) for r in range(world)]
    for pr in procs:
        pr.start()
    try:
        got = [out.get(timeout=300) for _ in range(world)]
    finally:
        for pr in procs:
            pr.join(timeout=60)
            if pr.is_alive():
                pr.terminate()
    assert all(pr.exitcode == 0 for pr in procs)
    got.sort(key=lambda g: g[1])                         # by first replica
    lp = lib_params(I, n, **kw)
    q = I.icd2s_qubo_create(Q)
    st = I.icd2s_state_create(q, kw["z"], seed)
    try:
        I.icd2s_initial_pass(st, lp)
        I.icd2s_best_update(st)
        whole = []
        for t in range(iters):
            I.icd2s_step(st, lp, t)
            whole.append(I.icd2s_get_state(st, kw["z"], n))
        wx, wE = I.icd2s_get_best(st, n)
    finally:
        I.icd2s_state_destroy(st)
        I.icd2s_qubo_destroy(q)
    torch.cuda.synchronize()
    o = orc.run(Q, orc_params(orc, lp), seed)
    z = kw["z"]
    for t in range(iters):
        xs = np.concatenate([g[2][t][0] for g in got])
        Es = np.concatenate([g[2][t][1] for g in got])
        assert np.array_equal(xs, whole[t][0]) and np.array_equal(Es, whole[t][2]), t
        assert np.array_equal(Es, o["trace"][t, 2 * z:3 * z]), t
    for rank, base, _, (E, r, bx) in got:               # every rank learns the same best
        assert E == wE == o["best_E"] and np.array_equal(bx, wx) and np.array_equal(bx, o["best_x"])
