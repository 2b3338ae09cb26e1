"""GPU parity at the library's size limits: the largest n (16 384, one row of
Q is 16 KiB and the Tabu kernel runs its widest shape), the most replicas
(4096), the largest subQUBO (256) and the longest schedule (16 384 sweeps,
a 256 MiB acceptance-limit table), each against the oracle; and the limits
themselves are rejected one step beyond them."""
import numpy as np
import pytest

from paper_2502_13947_gb300 import build as B
from paper_2502_13947_gb300 import icd2s as I
from paper_2502_13947_gb300.instances import make_qubo, random_solutions

from .gpu_util import dev, lib_params, orc_params, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    torch_cuda()
    B.build()
    return I.lib()


def _one_step(orc, Q, lp, seed, S0, t=0):
    n, z = Q.shape[0], lp.z
    q = I.icd2s_qubo_create(Q)
    st = I.icd2s_state_create(q, z, seed)
    try:
        I.icd2s_state_load(st, S0)
        I.icd2s_step(st, lp, t)
        x, g, E = I.icd2s_get_state(st, z, n)
        bx, bE = I.icd2s_get_best(st, n)
    finally:
        I.icd2s_state_destroy(st)
        I.icd2s_qubo_destroy(q)
    o = orc.step(Q, orc_params(orc, lp), seed, t, S0)
    assert np.array_equal(x, o["S"]) and np.array_equal(E, o["E"])
    assert bE == o["best_E"] and np.array_equal(bx, o["best_x"])
    return x, g


def test_largest_n_with_the_largest_subqubo(L, orc):
    """n = 16 384 (the maximum), one replica, a 256-variable subQUBO, the
    Eq. 5 mutation (r_0 = 0.6: thousands of flips through the split
    write-back)."""
    n = 16384
    Q = make_qubo(n, 1.0, 3)
    lp = lib_params(I, n, z=1, K=1, m_min=256, m_max=256, m_init=256, alpha=600, c=max(2, n // 150), sweeps=8,
                    T_max=2000.0, mut_mode=0, patience=0, max_iters=1)
    S0 = random_solutions(n, 1, 4)
    x, g = _one_step(orc, Q, lp, 17, S0)
    assert np.array_equal(g[0], orc.gains(Q, x[0]))


def test_most_replicas(L, orc):
    """4096 replicas (the maximum) of a small dense instance, uneven K = 2."""
    n, z = 64, 4096
    Q = make_qubo(n, 1.0, 8)
    lp = lib_params(I, n, z=z, K=2, m_min=5, m_max=12, m_init=12, alpha=2 * n, c=2, sweeps=16, T_max=300.0,
                    mut_mode=0, patience=0, max_iters=1)
    _one_step(orc, Q, lp, 5, random_solutions(n, z, 6), t=3)


def test_longest_schedule(L, orc):
    """16 384 sweeps (the maximum) on 8-variable subQUBOs."""
    torch = torch_cuda()
    n, R = 200, 2
    Q = make_qubo(n, 0.5, 12)
    q = I.icd2s_qubo_create(Q)
    st = I.icd2s_state_create(q, R, 2)
    X0 = random_solutions(n, R, 13)
    try:
        I.icd2s_state_load(st, X0)
        S = [np.sort(np.random.default_rng(p).choice(n, 8, replace=False)).astype(np.int32) for p in range(R)]
        idx_d, off_d = dev(np.concatenate(S)), dev(np.array([0, 8, 16], np.int32))
        mask = torch.zeros((R, n), dtype=torch.uint8, device="cuda")
        dE = torch.zeros(R, dtype=torch.int64, device="cuda")
        ap = I.AnnealParams(sweeps=16384, T_max=900.0, T_min=1.0, iter=4, per_replica=1)
        I.icd2s_anneal_subqubos_batch(st, idx_d.data_ptr(), off_d.data_ptr(), R, ap, mask.data_ptr(), dE.data_ptr())
        mask, dE = mask.cpu().numpy(), dE.cpu().numpy()
    finally:
        I.icd2s_state_destroy(st)
        I.icd2s_qubo_destroy(q)
    beta = orc.beta_table(16384, 900.0, 1.0)
    for p in range(R):
        Qs, _ = orc.subqubo(Q, X0[p], S[p])
        xs1, dEo, _ = orc.anneal(Qs, X0[p][S[p]], beta, orc.nlog_table(), 2, p, 4)
        assert dE[p] == dEo
        assert np.array_equal(mask[p][S[p]], (xs1 != X0[p][S[p]]).astype(np.uint8))


def test_one_beyond_each_limit_is_rejected(L):
    Q = make_qubo(64, 1.0, 1)
    q = I.icd2s_qubo_create(Q)
    try:
        with pytest.raises(I.ICD2SError) as e:
            I.icd2s_state_create(q, 4097, 1)
        assert e.value.code == I.ERR_RANGE
        st = I.icd2s_state_create(q, 2, 1)
        try:
            for kw in (dict(sweeps=16385), dict(m_min=257, m_max=257), dict(im_mode=1, m_min=25, m_max=25)):
                lp = lib_params(I, 64, z=2, K=1, m_min=16, m_max=16, m_init=16)
                for k, v in kw.items():
                    setattr(lp, k, v)
                with pytest.raises(I.ICD2SError):
                    I.icd2s_step(st, lp, 0)
        finally:
            I.icd2s_state_destroy(st)
    finally:
        I.icd2s_qubo_destroy(q)
    import ctypes
    h = ctypes.c_void_p()
    buf = np.zeros(16, np.int8)
    assert L.icd2s_qubo_create(buf.ctypes.data_as(ctypes.c_void_p), 16385, ctypes.byref(h)) == I.ERR_RANGE
