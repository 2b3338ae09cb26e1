"""GPU parity of whole trajectories: Algorithm 2 run by the library (through
the C ABI) equals the oracle's run bit for bit -- every energy after every
phase of every iteration, the final solutions and the best solution -- and a
full-size outer iteration of the n = 2500 workload equals the oracle's."""
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


def _compare_runs(orc, Q, lp, seed):
    q = I.icd2s_qubo_create(Q)
    try:
        g = I.icd2s_run(q, lp, seed, trace=True, want_S=True)
    finally:
        I.icd2s_qubo_destroy(q)
    o = orc.run(Q, orc_params(orc, lp), seed)
    assert g["iters"] == o["iters"]
    assert g["init_best_E"] == o["init_best_E"]
    assert np.array_equal(g["trace"], o["trace"])
    assert np.array_equal(g["S"], o["S"])
    assert g["best_E"] == o["best_E"] and np.array_equal(g["best_x"], o["best_x"])
    return g, o


def test_run_dense_n64_m16_z8_200_iterations(L, orc):
    """Dense n = 64, subQUBO 16, 8 replicas, 200 outer iterations x 256
    cosine-schedule sweeps, alpha = 5n, c = 2, the Eq. 5 mutation rate."""
    n = 64
    Q = make_qubo(n, 1.0, 2024)
    lp = lib_params(I, n, z=8, K=1, m_min=16, m_max=16, m_init=16, alpha=5 * n, c=2, sweeps=256,
                    T_max=600.0, T_min=1.0, mut_mode=0, patience=0, max_iters=200)
    g, o = _compare_runs(orc, Q, lp, 7)
    assert g["iters"] == 200
    assert g["anneal_attempts"] == 8 * (n // 16) * 256 * 16 + 200 * 8 * 256 * 16


def test_run_with_the_exact_ising_machine(L, orc):
    """Algorithm 2 with the exact Ising machine (im_mode 1): uneven K = 2
    subQUBOs of 6..12 variables, the initial pass on blocks of 12."""
    n = 64
    Q = make_qubo(n, 1.0, 77)
    lp = lib_params(I, n, z=4, K=2, m_min=6, m_max=12, m_init=12, alpha=3 * n, c=2, sweeps=8, T_max=500.0,
                    mut_mode=0, patience=0, max_iters=12, im_mode=1)
    _compare_runs(orc, Q, lp, 19)


@pytest.mark.parametrize("ablation", [1, 2])
def test_run_ablations(L, orc, ablation):
    """The simplified versions of Section 4: No_IM (1) and No_SM (2)."""
    n = 90
    Q = make_qubo(n, 0.6, 5 + ablation)
    lp = lib_params(I, n, z=5, K=2, m_min=7, m_max=12, m_init=12, alpha=2 * n, c=3, sweeps=16, T_max=300.0,
                    mut_mode=0, patience=0, max_iters=10, ablation=ablation)
    _compare_runs(orc, Q, lp, 23)


def test_run_with_aspiration(L, orc):
    n = 120
    Q = make_qubo(n, 0.4, 55)
    lp = lib_params(I, n, z=4, K=1, m_min=16, m_max=16, m_init=16, alpha=3 * n, c=40, sweeps=16, T_max=300.0,
                    mut_mode=0, patience=0, max_iters=8, aspiration=1)
    _compare_runs(orc, Q, lp, 31)


def test_run_with_patience_and_constant_rate(L, orc):
    n = 150
    Q = make_qubo(n, 0.3, 5)
    lp = lib_params(I, n, z=5, K=1, m_min=24, m_max=24, m_init=24, alpha=2 * n, c=3, sweeps=40, T_max=900.0,
                    mut_mode=1, mut_rate=0.05, patience=4, max_iters=300)
    g, o = _compare_runs(orc, Q, lp, 3)
    assert g["iters"] < 300


def test_run_batched_uneven_subqubos(L, orc):
    n = 600
    Q = make_qubo(n, 0.5, 8)
    lp = lib_params(I, n, z=3, K=6, m_min=8, m_max=70, m_init=37, alpha=n, c=4, sweeps=24, T_max=2000.0,
                    mut_mode=0, patience=0, max_iters=6)
    _compare_runs(orc, Q, lp, 11)


@pytest.mark.parametrize("scheme", [1, 2, 3, 4])
def test_run_uneven_subqubos_in_every_sweep_scheme(L, orc, scheme):
    """The persistent uneven-batch kernel (subQUBOs of 20..250 variables, all
    four lane layouts) in each sweep scheme: the whole run equals the
    oracle's."""
    n = 1200
    Q = make_qubo(n, 0.3, 9)
    lp = lib_params(I, n, z=3, K=4, m_min=20, m_max=250, m_init=100, alpha=n, c=4, sweeps=20, T_max=3000.0,
                    mut_mode=0, patience=0, max_iters=4)
    q = I.icd2s_qubo_create(Q)
    st = I.icd2s_state_create(q, lp.z, 13)
    try:
        I.icd2s_set_tuning(st, anneal_scheme=scheme)
        g = I.icd2s_state_run(st, n, lp, trace=True, want_S=True)
    finally:
        I.icd2s_state_destroy(st)
        I.icd2s_qubo_destroy(q)
    o = orc.run(Q, orc_params(orc, lp), 13)
    assert g["iters"] == o["iters"] and np.array_equal(g["trace"], o["trace"])
    assert np.array_equal(g["S"], o["S"])
    assert g["best_E"] == o["best_E"] and np.array_equal(g["best_x"], o["best_x"])


def test_run_tiny_instances_reach_the_optimum(L, orc):
    import itertools
    for n, seed in [(12, 1), (16, 2)]:
        Q = make_qubo(n, 1.0, seed)
        X = np.array(list(itertools.product([0, 1], repeat=n)), dtype=np.int64)
        opt = int(np.einsum("ki,ij,kj->k", X, Q.astype(np.int64), X).min())
        lp = lib_params(I, n, z=4, m_min=4, m_max=4, m_init=4, sweeps=64, T_max=300.0, patience=0, max_iters=30)
        g, _ = _compare_runs(orc, Q, lp, 1000 + seed)
        assert g["best_E"] == opt


@pytest.mark.slow
def test_full_size_step_n2500_density01_m64_z128(L, orc):
    """One whole outer iteration at the benchmark's sizes (n = 2500, 10 %
    density, subQUBO 64, 128 replicas, 1024 sweeps, alpha = 5n, c = 16,
    mutation rate 1 %), launched exactly as the benchmark launches it."""
    n, z = 2500, 128
    Q = make_qubo(n, 0.1, 1)
    lp = lib_params(I, n, z=z, K=1, m_min=64, m_max=64, m_init=64, alpha=5 * n, c=16, sweeps=1024,
                    T_max=1500.0, T_min=1.0, mut_mode=1, mut_rate=0.01)
    S0 = random_solutions(n, z, 42)
    q = I.icd2s_qubo_create(Q)
    st = I.icd2s_state_create(q, z, 9)
    try:
        I.icd2s_state_load(st, S0)
        I.icd2s_step(st, lp, 0)
        x, g, E = I.icd2s_get_state(st, z, n)
        bx, bE = I.icd2s_get_best(st, n)
    finally:
        I.icd2s_state_destroy(st)
        I.icd2s_qubo_destroy(q)
    o = orc.step(Q, orc_params(orc, lp), 9, 0, S0)
    assert np.array_equal(x, o["S"])
    assert np.array_equal(E, o["E"])
    assert bE == o["best_E"] and np.array_equal(bx, o["best_x"])
    for p in range(0, z, 16):      # gains: a sample of replicas, each against its definition
        assert np.array_equal(g[p], orc.gains(Q, x[p]))


# ----------------------------------------------------------------------------- CUDA graph replay
@pytest.mark.parametrize("K,m_min,m_max,patience", [(1, 16, 16, 0), (4, 8, 40, 0), (3, 10, 30, 5)])
def test_graph_replayed_run_matches_the_oracle(L, orc, K, m_min, m_max, patience):
    """One outer iteration captured as a CUDA graph and replayed (the
    iteration number and mutation rate read from device memory); uneven
    batches go through the persistent queue kernel."""
    n = 200
    Q = make_qubo(n, 0.6, 31)
    lp = lib_params(I, n, z=5, K=K, m_min=m_min, m_max=m_max, m_init=m_max, alpha=n, c=3, sweeps=32,
                    T_max=1200.0, mut_mode=0, patience=patience, max_iters=25, use_graph=1)
    q = I.icd2s_qubo_create(Q)
    try:
        g = I.icd2s_run(q, lp, 17, trace=False, want_S=True)
    finally:
        I.icd2s_qubo_destroy(q)
    o = orc.run(Q, orc_params(orc, lp), 17)
    assert g["iters"] == o["iters"]
    assert np.array_equal(g["S"], o["S"])
    assert g["best_E"] == o["best_E"] and np.array_equal(g["best_x"], o["best_x"])


def test_graph_steps_equal_plain_steps_on_a_stream(L):
    torch = torch_cuda()
    n, z = 500, 6
    Q = make_qubo(n, 0.3, 3)
    q = I.icd2s_qubo_create(Q)
    S0 = random_solutions(n, z, 5)
    out = []
    for use_graph in (0, 1):
        lp = lib_params(I, n, z=z, K=3, m_min=12, m_max=70, m_init=50, alpha=n, c=4, sweeps=20, T_max=900.0,
                        use_graph=use_graph)
        st = I.icd2s_state_create(q, z, 3)
        s = torch.cuda.Stream()
        I.icd2s_state_load(st, S0, stream=s.cuda_stream)
        for t in (0, 1, 2, 7, 8):   # a jump in t re-seeds the device iteration number
            I.icd2s_step(st, lp, t, s.cuda_stream)
        s.synchronize()
        out.append(I.icd2s_get_state(st, z, n))
        I.icd2s_state_destroy(st)
    I.icd2s_qubo_destroy(q)
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("im_mode,K,m_min,m_max", [(0, 6, 8, 70), (0, 4, 20, 250), (1, 3, 6, 12)])
def test_run_gauss_seidel_subqubos(L, orc, im_mode, K, m_min, m_max):
    """im_order 1: a solution's subQUBOs are annealed (or solved exactly) one
    group at a time, each built from the solution the earlier groups left;
    the whole run (replayed as a CUDA graph) equals the oracle's."""
    n = 1100
    Q = make_qubo(n, 0.4, 12)
    # a short Tabu search leaves the solutions far from a local minimum, so the
    # Ising machine changes many variables and the order of the groups matters
    lp = lib_params(I, n, z=3, K=K, m_min=m_min, m_max=m_max, m_init=min(m_max, 64), alpha=5, c=4,
                    sweeps=20, T_max=2500.0, mut_mode=0, patience=0, max_iters=4, im_mode=im_mode, im_order=1)
    g, o = _compare_runs(orc, Q, lp, 19)
    lp.im_order = 0
    q = I.icd2s_qubo_create(Q)
    try:
        j = I.icd2s_run(q, lp, 19, trace=True)
    finally:
        I.icd2s_qubo_destroy(q)
    assert not np.array_equal(j["trace"], g["trace"])  # the order matters on this instance


def test_run_with_a_move_log_beyond_shared_memory(L, orc):
    """A whole run (replayed as a CUDA graph) whose Tabu searches keep their
    move logs in global memory: alpha = 400 n at n = 300."""
    n = 300
    Q = make_qubo(n, 0.5, 44)
    lp = lib_params(I, n, z=2, K=1, m_min=32, m_max=32, m_init=32, alpha=400 * n, c=5, sweeps=16,
                    T_max=1500.0, mut_mode=0, patience=0, max_iters=2)
    _compare_runs(orc, Q, lp, 45)


@pytest.mark.parametrize("n,K,use_graph,G", [(2400, 4, 1, 2), (4200, 1, 0, 4), (8300, 2, 1, 0)])
def test_run_with_the_tabu_search_split_over_clusters(L, orc, n, K, use_graph, G):
    """Few replicas of a large instance with each replica's Tabu search split
    over a cluster of 2 or 4 CTAs (n = 8300: the default split, 4); the whole
    run (two of them replayed as a CUDA graph) equals the oracle's."""
    Q = make_qubo(n, 0.3, 23)
    lp = lib_params(I, n, z=3, K=K, m_min=16, m_max=64, m_init=64, alpha=n, c=max(2, n // 150), sweeps=16,
                    T_max=2000.0, mut_mode=0, patience=0, max_iters=3 if n < 8000 else 2, use_graph=use_graph)
    q = I.icd2s_qubo_create(Q)
    st = I.icd2s_state_create(q, lp.z, 29)
    try:
        I.icd2s_set_tuning(st, tabu_cluster=G)
        g = I.icd2s_state_run(st, n, lp, trace=True, want_S=True)
    finally:
        I.icd2s_state_destroy(st)
        I.icd2s_qubo_destroy(q)
    o = orc.run(Q, orc_params(orc, lp), 29)
    assert g["iters"] == o["iters"] and np.array_equal(g["trace"], o["trace"])
    assert np.array_equal(g["S"], o["S"])
    assert g["best_E"] == o["best_E"] and np.array_equal(g["best_x"], o["best_x"])


@pytest.mark.parametrize("K,m_min,m_max", [(1, 32, 32), (3, 10, 60)])
def test_im_round_equals_its_pieces(L, orc, K, m_min, m_max):
    """icd2s_im_round (selection, one batched anneal launch, write-back, all
    on the device) equals the same round made of the separately
    oracle-checked calls: icd2s_select_subqubos, icd2s_anneal_subqubos_batch
    and icd2s_apply_flips_update_gains; and the tracked gains stay exact (a
    tensor-core refresh finds no difference)."""
    torch = torch_cuda()
    n, R, t = 600, 4, 3
    Q = make_qubo(n, 0.5, 5)
    X0 = random_solutions(n, R, 6)
    lp = lib_params(I, n, z=R, K=K, m_min=m_min, m_max=m_max, m_init=m_max, alpha=n, c=4, sweeps=32,
                    T_max=2000.0)
    q = I.icd2s_qubo_create(Q)
    a = I.icd2s_state_create(q, R, 8)
    b = I.icd2s_state_create(q, R, 8)
    try:
        for st in (a, b):
            I.icd2s_state_load(st, X0)
            I.icd2s_tabu(st, lp.alpha, lp.c)
        I.icd2s_im_round(a, lp, t)
        idx = torch.zeros(R * K * m_max + 1, dtype=torch.int32, device="cuda")
        off = torch.zeros(R * K * m_max + 1, dtype=torch.int32, device="cuda")
        mask = torch.zeros((R, n), dtype=torch.uint8, device="cuda")
        I.icd2s_select_subqubos(b, I.SelectParams(w1=lp.w1, w2=lp.w2, w3=lp.w3, K=K, m_min=m_min, m_max=m_max,
                                                  iter=t), idx.data_ptr(), off.data_ptr())
        I.icd2s_anneal_subqubos_batch(b, idx.data_ptr(), off.data_ptr(), R * K,
                                      I.AnnealParams(sweeps=lp.sweeps, T_max=lp.T_max, T_min=lp.T_min, iter=t,
                                                     per_replica=K), mask.data_ptr())
        I.icd2s_apply_flips_update_gains(b, mask.data_ptr())
        sa, sb = I.icd2s_get_state(a, R, n), I.icd2s_get_state(b, R, n)
        for u, v in zip(sa, sb):
            assert np.array_equal(u, v)
        assert not np.array_equal(sa[0], X0)          # the round changed the solutions
        assert I.icd2s_refresh(a) == 0
        assert np.array_equal(sa[2], orc.energy_batch(Q, sa[0]))
    finally:
        I.icd2s_state_destroy(a)
        I.icd2s_state_destroy(b)
        I.icd2s_qubo_destroy(q)
