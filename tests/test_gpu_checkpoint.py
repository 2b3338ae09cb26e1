"""Checkpoint and resume on the GPU.  A run stopped after iteration t - 1,
saved, restored into a fresh state (created with another seed, which the
checkpoint's replaces) and resumed at t gives the uninterrupted run's
trajectory, final solutions and best solution bit for bit: the plain method
(the joined trajectory also equal to the oracle's), the learned selection
(hit counts carried over), patience termination (the stale count carried
over) and CUDA-graph replay.  A save/restore round trip keeps solutions,
gains, energies, best solution and hit counts; a damaged or mismatched
checkpoint is refused and leaves the state as it was."""
import numpy as np
import pytest

from paper_2502_13947_gb300 import build as B
from paper_2502_13947_gb300 import icd2s as I
from paper_2502_13947_gb300.instances import make_qubo

from .gpu_util import lib_params, orc_params, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    torch_cuda()
    B.build()
    return I.lib()


def _params(lp, **kw):
    p = I.Params.from_buffer_copy(lp)
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def _state(q, z, seed, mlp):
    st = I.icd2s_state_create(q, z, seed)
    if mlp is not None:
        I.icd2s_state_set_mlp(st, mlp)
    return st


def _whole(Q, lp, seed, mlp=None, trace=True):
    n = Q.shape[0]
    q = I.icd2s_qubo_create(Q)
    st = _state(q, lp.z, seed, mlp)
    try:
        return I.icd2s_state_run(st, n, lp, trace=trace, want_S=True)
    finally:
        I.icd2s_state_destroy(st)
        I.icd2s_qubo_destroy(q)


def _resumed(Q, lp, seed, split, mlp=None, trace=True, graph=0):
    """Runs iterations 0 .. split - 1, saves, restores into a new state and
    runs the rest; returns the second part with the first part's trace rows."""
    n = Q.shape[0]
    q = I.icd2s_qubo_create(Q)
    try:
        st = _state(q, lp.z, seed, mlp)
        try:
            first = I.icd2s_state_run(st, n, _params(lp, max_iters=split), trace=trace, want_S=True)
            blob = I.icd2s_state_save(st, first["iters"])
        finally:
            I.icd2s_state_destroy(st)
        assert I.icd2s_checkpoint_info(blob) == (n, lp.z, first["iters"], seed)
        st = _state(q, lp.z, seed + 1000, mlp)
        try:
            t = I.icd2s_state_restore(st, blob)
            assert t == first["iters"]
            second = I.icd2s_state_run(st, n, _params(lp, t_start=t, use_graph=graph), trace=trace and not graph,
                                       want_S=True)
        finally:
            I.icd2s_state_destroy(st)
    finally:
        I.icd2s_qubo_destroy(q)
    if trace and not graph:
        second["trace"][:t] = first["trace"][:t]
    return first, second


def _same(a, b, trace=True):
    assert a["iters"] == b["iters"]
    assert a["best_E"] == b["best_E"] and np.array_equal(a["best_x"], b["best_x"])
    assert np.array_equal(a["S"], b["S"])
    if trace:
        assert np.array_equal(a["trace"], b["trace"])


def test_resumed_plain_run_equals_the_uninterrupted_run_and_the_oracle(L, orc):
    n, seed = 120, 4
    Q = make_qubo(n, 0.5, 31)
    lp = lib_params(I, n, z=6, K=2, m_min=8, m_max=20, m_init=20, alpha=2 * n, c=3, sweeps=32, T_max=400.0,
                    mut_mode=0, patience=0, max_iters=12)
    whole = _whole(Q, lp, seed)
    o = orc.run(Q, orc_params(orc, lp), seed)
    assert np.array_equal(whole["trace"], o["trace"]) and whole["best_E"] == o["best_E"]
    for split in (1, 5, 11, 12):
        _, resumed = _resumed(Q, lp, seed, split)
        _same(whole, resumed)
        assert np.array_equal(resumed["trace"], o["trace"]), split


def test_resumed_learned_run_carries_the_hit_counts(L):
    n, seed = 130, 9
    Q = make_qubo(n, 0.7, 12)
    lp = lib_params(I, n, z=4, K=1, m_min=16, m_max=16, m_init=16, alpha=n, c=2, sweeps=24, T_max=300.0,
                    mut_mode=0, patience=0, max_iters=10, select_mode=2)
    m = I.icd2s_mlp_create(3)
    try:
        whole = _whole(Q, lp, seed, mlp=m)
        _, resumed = _resumed(Q, lp, seed, 6, mlp=m)
        _same(whole, resumed)
    finally:
        I.icd2s_mlp_destroy(m)


def test_resumed_run_stops_by_patience_where_the_uninterrupted_run_does(L):
    n, seed = 100, 2
    Q = make_qubo(n, 0.6, 8)
    lp = lib_params(I, n, z=4, K=1, m_min=12, m_max=12, m_init=12, alpha=n, c=2, sweeps=16, T_max=200.0,
                    mut_mode=1, mut_rate=0.02, patience=3, max_iters=80)
    whole = _whole(Q, lp, seed)
    assert 3 <= whole["iters"] < 80
    split = max(1, whole["iters"] - 2)  # inside the final stale stretch when that is long enough
    first, resumed = _resumed(Q, lp, seed, split)
    assert first["iters"] == split
    _same(whole, resumed)


def test_resumed_run_with_graph_replay(L):
    n, seed = 96, 5
    Q = make_qubo(n, 0.5, 44)
    lp = lib_params(I, n, z=4, K=2, m_min=8, m_max=16, m_init=16, alpha=n, c=2, sweeps=16, T_max=300.0,
                    mut_mode=0, patience=0, max_iters=9)
    whole = _whole(Q, lp, seed, trace=False)
    _, resumed = _resumed(Q, lp, seed, 4, trace=False, graph=1)
    _same(whole, resumed, trace=False)


def test_round_trip_and_refusals_leave_the_state_unchanged(L):
    n, z, seed = 77, 3, 6
    Q = make_qubo(n, 0.5, 3)
    lp = lib_params(I, n, z=z, K=1, m_min=10, m_max=10, m_init=10, alpha=n, c=2, sweeps=16, T_max=300.0,
                    mut_mode=0, patience=0, max_iters=3)
    q = I.icd2s_qubo_create(Q)
    sts = []
    try:
        a = I.icd2s_state_create(q, z, seed)
        sts.append(a)
        I.icd2s_state_run(a, n, lp)
        blob = I.icd2s_state_save(a, 3)
        assert len(blob) == 72 + 5 * z * n + n
        b = I.icd2s_state_create(q, z, seed + 1)
        sts.append(b)
        before = I.icd2s_get_state(b, z, n)
        bad = bytearray(blob)
        bad[64 + 5] ^= 1
        with pytest.raises(I.ICD2SError) as e:
            I.icd2s_state_restore(b, bytes(bad))
        assert e.value.code == I.ERR_INVARIANT
        c = I.icd2s_state_create(q, z + 1, seed)
        sts.append(c)
        with pytest.raises(I.ICD2SError) as e:
            I.icd2s_state_restore(c, blob)
        assert e.value.code == I.ERR_ARG
        after = I.icd2s_get_state(b, z, n)
        assert all(np.array_equal(u, v) for u, v in zip(before, after))
        assert I.icd2s_state_restore(b, blob) == 3
        for u, v in zip(I.icd2s_get_state(a, z, n), I.icd2s_get_state(b, z, n)):
            assert np.array_equal(u, v)  # gains and energies recomputed equal the tracked ones
        xa, Ea = I.icd2s_get_best(a, n)
        xb, Eb = I.icd2s_get_best(b, n)
        assert Ea == Eb and np.array_equal(xa, xb)
        assert np.array_equal(I.icd2s_get_hits(a, z, n), I.icd2s_get_hits(b, z, n))
        assert I.icd2s_state_save(b, 3) == blob
        with pytest.raises(I.ICD2SError) as e:
            I.icd2s_state_run(b, n, _params(lp, t_start=4))
        assert e.value.code == I.ERR_ARG
        with pytest.raises(I.ICD2SError) as e:
            I.icd2s_run(q, _params(lp, t_start=1), seed)
        assert e.value.code == I.ERR_ARG
    finally:
        for st in sts:
            I.icd2s_state_destroy(st)
        I.icd2s_qubo_destroy(q)
