"""GPU parity of the replica-sharded path: a solution set split into replica
shards (each its own state, as each GPU of a multi-GPU run holds one), with
the shards' column counts added between the two halves of every outer
iteration, evolves exactly like the whole set on one state and like the
oracle's run (Algorithm 2).  The ranks are emulated in one process on one
GPU: the counts are added on the device between calls, and no kernel waits
on another shard's."""
import numpy as np
import pytest

from paper_2502_13947_gb300 import build as B
from paper_2502_13947_gb300 import icd2s as I
from paper_2502_13947_gb300.instances import make_qubo
from paper_2502_13947_gb300.shard import shard_range

from .gpu_util import lib_params, orc_params, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    torch_cuda()
    B.build()
    return I.lib()


def _run_shards(Q, lp, seed, world, iters):
    """Runs `iters` iterations on `world` shards; returns the concatenated
    solutions and energies after each iteration and the best over shards."""
    torch = torch_cuda()
    n, z = Q.shape[0], lp.z
    q = I.icd2s_qubo_create(Q)
    shards = [I.icd2s_state_create_shard(q, c, b, z, seed)
              for b, c in (shard_range(z, r, world) for r in range(world))]
    counts = [torch.zeros(n, dtype=torch.int32, device="cuda") for _ in shards]
    total = torch.zeros(n, dtype=torch.int32, device="cuda")
    per_iter = []
    try:
        for st in shards:
            I.icd2s_initial_pass(st, lp)
            I.icd2s_best_update(st)
        for t in range(iters):
            for st, c in zip(shards, counts):
                I.icd2s_step_shard_begin(st, lp, t, c.data_ptr())
            torch.sum(torch.stack(counts), dim=0, dtype=torch.int32, out=total)   # the allreduce
            for st in shards:
                I.icd2s_step_shard_finish(st, lp, t, total.data_ptr())
            parts = [I.icd2s_get_state(st, c, n) for st, c in
                     zip(shards, (shard_range(z, r, world)[1] for r in range(world)))]
            per_iter.append((np.concatenate([x for x, _, _ in parts]), np.concatenate([E for _, _, E in parts])))
        infos = [I.icd2s_get_best_info(st) for st in shards]
        k = min(range(world), key=lambda r: (infos[r][0], infos[r][2], infos[r][1]))
        best = (infos[k][0], infos[k][1], I.icd2s_get_best(shards[k], n)[0])
    finally:
        for st in shards:
            I.icd2s_state_destroy(st)
        I.icd2s_qubo_destroy(q)
    return per_iter, best


def _run_whole(Q, lp, seed, iters):
    n, z = Q.shape[0], lp.z
    q = I.icd2s_qubo_create(Q)
    st = I.icd2s_state_create(q, z, seed)
    per_iter = []
    try:
        I.icd2s_initial_pass(st, lp)
        I.icd2s_best_update(st)
        for t in range(iters):
            I.icd2s_step(st, lp, t)
            x, _, E = I.icd2s_get_state(st, z, n)
            per_iter.append((x, E))
        bx, bE = I.icd2s_get_best(st, n)
    finally:
        I.icd2s_state_destroy(st)
        I.icd2s_qubo_destroy(q)
    return per_iter, (bE, bx)


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("case", ["plain", "uneven batch", "No_SM", "Gauss-Seidel", "aspiration"])
def test_shards_evolve_like_the_whole_set_and_the_oracle(L, orc, world, case):
    n, iters, seed = 300, 4, 21
    Q = make_qubo(n, 0.5, 17)
    kw = dict(z=6, K=1, m_min=24, m_max=24, m_init=24, alpha=n, c=3, sweeps=24, T_max=1500.0, mut_mode=0,
              patience=0, max_iters=iters)
    if case == "uneven batch":
        kw.update(K=4, m_min=8, m_max=40, m_init=32)
    if case == "No_SM":
        kw.update(ablation=2)
    if case == "Gauss-Seidel":
        kw.update(K=3, m_min=10, m_max=30, m_init=30, im_order=1)
    if case == "aspiration":
        kw.update(aspiration=1, c=40)
    lp = lib_params(I, n, **kw)
    sh, (sE, sr, sx) = _run_shards(Q, lp, seed, world, iters)
    wh, (wE, wx) = _run_whole(Q, lp, seed, iters)
    for t in range(iters):
        assert np.array_equal(sh[t][0], wh[t][0]), t
        assert np.array_equal(sh[t][1], wh[t][1]), t
    assert sE == wE and np.array_equal(sx, wx)
    o = orc.run(Q, orc_params(orc, lp), seed)
    z = lp.z
    for t in range(iters):     # the energies after each iteration's mutation, per replica
        assert np.array_equal(sh[t][1], o["trace"][t, 2 * z:3 * z]), t
    assert np.array_equal(sh[-1][0], o["S"])
    assert sE == o["best_E"] and np.array_equal(sx, o["best_x"])


def test_a_shard_refuses_the_whole_set_calls(L):
    n = 200
    Q = make_qubo(n, 0.5, 3)
    q = I.icd2s_qubo_create(Q)
    st = I.icd2s_state_create_shard(q, 2, 2, 5, 1)
    lp = lib_params(I, n, z=5, K=1, m_min=16, m_max=16, m_init=16, alpha=n, c=3, sweeps=8, T_max=900.0)
    try:
        with pytest.raises(I.ICD2SError) as e:
            I.icd2s_step(st, lp, 0)
        assert e.value.code == I.ERR_STATE
        with pytest.raises(I.ICD2SError):
            I.icd2s_state_create_shard(q, 3, 3, 5, 1)     # replicas 3..5 of 5
    finally:
        I.icd2s_state_destroy(st)
        I.icd2s_qubo_destroy(q)
