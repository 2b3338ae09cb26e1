"""Out-of-memory paths on the GPU, made on the host with the library's
allocation hook (no real exhaustion of device memory).  A job that touches
every lazily made buffer -- instance, network, state, improvement log,
mutation rates, temperature tables, features and scores, the tensor-core
refresh operands and results, signed rows, a Tabu move log in global memory
-- is run once with each of its device allocations failing in turn: the
failing call reports ICD2S_ERR_OOM, the same call succeeds once the hook is
off, and the job ends with the results of a run that never failed (buffers
that belong together are made all or none, and no failed allocation leaves a
pending error behind for a later launch check)."""
import numpy as np
import pytest

from paper_2502_13947_gb300 import build as B
from paper_2502_13947_gb300 import icd2s as I
from paper_2502_13947_gb300.instances import make_qubo

from .gpu_util import lib_params, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    torch_cuda()
    B.build()
    return I.lib()


def _job(Q, lp, seed, fail_at):
    """Returns (results, number of OOM failures met)."""
    n = Q.shape[0]
    failures = 0

    def call(fn, *args, **kw):
        nonlocal failures
        while True:
            try:
                return fn(*args, **kw)
            except I.ICD2SError as e:
                assert e.code == I.ERR_OOM, e
                assert fail_at is not None
                failures += 1
                I.icd2s_debug_fail_allocations_after(-1)  # memory is back: the retry must succeed

    q = m = st = None
    out = {}
    if fail_at is not None:
        I.icd2s_debug_fail_allocations_after(fail_at)
    try:
        q = call(I.icd2s_qubo_create, Q)
        m = call(I.icd2s_mlp_create, 5)
        st = call(I.icd2s_state_create, q, lp.z, seed)
        x0 = I.icd2s_get_state(st, lp.z, n)[0]
        call(I.icd2s_state_set_mlp, st, m)
        call(I.icd2s_log_enable, st, 2)

        def run():
            I.icd2s_state_load(st, x0)  # a retry starts from the same solutions
            return I.icd2s_state_run(st, n, lp, trace=True, want_S=True)

        r = call(run)
        out["trace"], out["S"], out["best_E"] = r["trace"], r["S"], r["best_E"]
        call(I.icd2s_set_tuning, st, tabu_rows=2)

        def tabu():
            I.icd2s_state_load(st, r["S"])
            I.icd2s_tabu(st, 120000, 2)  # 2 bytes a move: the log goes to global memory
            return I.icd2s_get_state(st, lp.z, n)

        out["tabu"] = call(tabu)
    finally:
        I.icd2s_debug_fail_allocations_after(-1)
        if st is not None:
            I.icd2s_state_destroy(st)
        if m is not None:
            I.icd2s_mlp_destroy(m)
        if q is not None:
            I.icd2s_qubo_destroy(q)
    return out, failures


def test_each_allocation_failing_in_turn(L):
    n, seed = 100, 3
    Q = make_qubo(n, 0.5, 21)
    lp = lib_params(I, n, z=4, K=2, m_min=8, m_max=16, m_init=16, alpha=n, c=2, sweeps=16, T_max=300.0,
                    mut_mode=0, patience=0, max_iters=4, refresh_every=2, select_mode=2)
    ref, f = _job(Q, lp, seed, None)
    assert f == 0
    k = 0
    while True:
        out, f = _job(Q, lp, seed, k)
        assert f <= 1
        assert np.array_equal(out["trace"], ref["trace"]) and np.array_equal(out["S"], ref["S"]), k
        assert out["best_E"] == ref["best_E"], k
        for a, b in zip(out["tabu"], ref["tabu"]):
            assert np.array_equal(a, b), k
        if f == 0:
            break
        k += 1
    assert k >= 40, k  # the job's device allocations, each of which failed once
