"""GPU parity of the dense refresh (tcgen05, BF16 operands, FP32 accumulation):
the recomputed gains and energies of every replica equal the oracle's
definition-level values, and equal the incrementally tracked ones after any
number of steps (the drift check reports zero differences)."""
import numpy as np
import pytest

from paper_2502_13947_gb300 import build as B
from paper_2502_13947_gb300 import icd2s as I
from paper_2502_13947_gb300.instances import make_qubo, random_solutions

from .gpu_util import lib_params, orc_params, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    torch_cuda()
    B.build()
    return I.lib()


@pytest.mark.parametrize("kind", [1, 3, 4])
@pytest.mark.parametrize("n,R,density", [(1, 1, 1.0), (64, 8, 1.0), (200, 16, 0.5), (300, 5, 0.3),
                                         (1000, 33, 1.0), (2500, 130, 0.1), (4097, 3, 1.0)])
def test_refresh_equals_the_definition(L, orc, n, R, density, kind):
    """Every operand path: BF16 copies of Q and X loaded by TMA (tiles of 128
    or 256 rows of Q, persistent over the SMs), and Q's bytes converted to BF16
    in shared memory."""
    Q = make_qubo(n, density, n + R)
    X = random_solutions(n, R, 4)
    q = I.icd2s_qubo_create(Q)
    st = I.icd2s_state_create(q, R, 1)
    try:
        I.icd2s_set_tuning(st, refresh_kind=kind)
        I.icd2s_state_load(st, X)
        assert I.icd2s_refresh(st) == 0          # tracked (dp4a recompute) == tensor-core recompute
        assert I.icd2s_refresh(st, rebuild=True) == 0
        x, g, E = I.icd2s_get_state(st, R, n)
    finally:
        I.icd2s_state_destroy(st)
        I.icd2s_qubo_destroy(q)
    assert np.array_equal(E, orc.energy_batch(Q, X))
    for p in range(0, R, max(1, R // 6)):
        assert np.array_equal(g[p], orc.gains(Q, X[p]))


def test_refresh_after_steps_dense_n7000_R256(L, orc):
    """The dense workload: n = 7000, every entry present, 256 replicas.  After
    outer iterations the tracked state still equals a from-scratch recompute
    (all 256 x 7000 gains and 256 energies), and sampled replicas equal the
    oracle's definition."""
    n, R = 7000, 256
    Q = make_qubo(n, 1.0, 7)
    q = I.icd2s_qubo_create(Q)
    st = I.icd2s_state_create(q, R, 3)
    lp = lib_params(I, n, z=R, K=4, m_min=32, m_max=256, m_init=64, alpha=200, c=46, sweeps=16,
                    T_max=5000.0, mut_mode=1, mut_rate=0.01)
    try:
        for t in range(2):
            I.icd2s_step(st, lp, t)
        for kind in (1, 3, 4):
            for bn, splits in ((256, 0), (128, 1), (256, 3), (128, 0), (256, 151)):
                I.icd2s_set_tuning(st, refresh_bn=bn, refresh_splits=splits, refresh_kind=kind)
                assert I.icd2s_refresh(st) == 0, (kind, bn, splits)
        x, g, E = I.icd2s_get_state(st, R, n)
    finally:
        I.icd2s_state_destroy(st)
        I.icd2s_qubo_destroy(q)
    for p in (0, 101, 255):
        assert E[p] == orc.energy(Q, x[p])
        assert np.array_equal(g[p], orc.gains(Q, x[p]))


def test_run_with_periodic_refresh_matches_the_oracle(L, orc):
    n = 300
    Q = make_qubo(n, 0.5, 2)
    lp = lib_params(I, n, z=6, K=2, m_min=10, m_max=40, m_init=30, alpha=n, c=3, sweeps=24, T_max=1500.0,
                    patience=0, max_iters=12, refresh_every=4)
    q = I.icd2s_qubo_create(Q)
    try:
        g = I.icd2s_run(q, lp, 9, trace=True, want_S=True)
    finally:
        I.icd2s_qubo_destroy(q)
    o = orc.run(Q, orc_params(orc, lp), 9)
    assert np.array_equal(g["trace"], o["trace"]) and np.array_equal(g["S"], o["S"])


@pytest.mark.parametrize("kind", [1, 3, 4])
def test_refresh_wait_timeout_is_reported_and_the_state_stays_usable(L, orc, kind):
    """Failure detection on the device: a refresh whose producer issues no
    loads (fault injection) has every tensor-core pipeline wait run out after
    2 ms; the kernel raises its flag, frees its tensor memory and returns,
    icd2s_refresh returns ICD2S_ERR_TIMEOUT without rebuilding from the
    incomplete sums, and the next refresh on the same state is exact."""
    n, R = 1000, 33
    Q = make_qubo(n, 1.0, 12)
    X = random_solutions(n, R, 13)
    q = I.icd2s_qubo_create(Q)
    st = I.icd2s_state_create(q, R, 1)
    try:
        I.icd2s_set_tuning(st, refresh_kind=kind)
        I.icd2s_state_load(st, X)
        assert I.icd2s_refresh(st) == 0
        I.icd2s_debug_refresh_stall(st, 1, 2000)
        with pytest.raises(I.ICD2SError) as e:
            I.icd2s_refresh(st, rebuild=True)
        assert e.value.code == I.ERR_TIMEOUT
        x, g, E = I.icd2s_get_state(st, R, n)       # the tracked values were not replaced
        assert np.array_equal(E, orc.energy_batch(Q, X))
        assert np.array_equal(g[5], orc.gains(Q, X[5]))
        assert I.icd2s_refresh(st) == 0             # the next refresh runs normally
        assert I.icd2s_refresh(st, rebuild=True) == 0
    finally:
        I.icd2s_state_destroy(st)
        I.icd2s_qubo_destroy(q)
