"""Pins of the oracle's method steps (Algorithms 1-4, Eq. 4-8, the mutation
operator and the whole loop) against hand-worked examples, brute force on
tiny inputs, closed forms and invariants.  No GPU."""
import itertools
import json
import math
import os

import numpy as np
import pytest

from paper_2502_13947_gb300.instances import make_qubo, random_solutions, random_subsets

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _gold(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def brute_min(Q):
    n = Q.shape[0]
    X = np.array(list(itertools.product([0, 1], repeat=n)), dtype=np.int64)
    E = np.einsum("ki,ij,kj->k", X, Q.astype(np.int64), X)
    return int(E.min()), X[E == E.min()].astype(np.uint8)


def full_energy(Q, x):
    x = x.astype(np.int64)
    return int(x @ Q.astype(np.int64) @ x)


# ----------------------------------------------------------------------------- Algorithm 1
def test_tabu_hand_worked_example(orc):
    g = _gold("tabu3_worked.json")
    Q = np.array(g["Q"], dtype=np.int8)
    x, E, T, C = orc.tabu(Q, np.array(g["x0"], np.uint8), g["alpha"], g["c"])
    assert x.tolist() == g["x_min"] and E == g["E_min"]
    assert T.tolist() == g["T"] and C.tolist() == g["C"]


def _tabu_by_full_energies(Q, x, alpha, c):
    """Algorithm 1 evaluated with whole-energy differences instead of the
    incremental move values (brute force; tiny n only)."""
    n = Q.shape[0]
    x = x.copy()
    C = np.zeros(n, np.int64)
    T = np.zeros(n, np.int64)
    OV = full_energy(Q, x)
    best, xbest = OV, x.copy()
    for _ in range(alpha):
        moves = []
        for k in range(n):
            if C[k] <= 0:
                y = x.copy()
                y[k] ^= 1
                moves.append((full_energy(Q, y) - OV, k))
        d, i = min(moves)
        OV += d
        x[i] ^= 1
        T[i] += 1
        C[i] += c
        C[C > 0] -= 1
        if OV < best:
            best, xbest = OV, x.copy()
    return xbest, best, T, C


@pytest.mark.parametrize("n,alpha,c,seed", [(12, 40, 2, 1), (14, 60, 5, 2), (9, 30, 1, 3), (16, 80, 3, 4)])
def test_tabu_matches_whole_energy_brute_force(orc, n, alpha, c, seed):
    Q = make_qubo(n, 1.0, seed)
    for x0 in random_solutions(n, 3, seed):
        xo, Eo, To, Co = orc.tabu(Q, x0, alpha, c)
        xb, Eb, Tb, Cb = _tabu_by_full_energies(Q, x0, alpha, c)
        assert Eo == Eb and np.array_equal(xo, xb)
        assert np.array_equal(To, Tb) and np.array_equal(Co, Cb)
        assert Eo == orc.energy(Q, xo)


def test_tabu_single_iteration_takes_the_best_move(orc):
    Q = make_qubo(50, 0.5, 8)
    for x0 in random_solutions(50, 5, 8):
        g = orc.gains(Q, x0)
        i = int(np.argmin(g))  # numpy argmin returns the lowest index on ties
        x, E, T, C = orc.tabu(Q, x0, 1, 2)
        E0 = orc.energy(Q, x0)
        assert T.tolist() == [1 if k == i else 0 for k in range(50)]
        if g[i] < 0:
            y = x0.copy()
            y[i] ^= 1
            assert np.array_equal(x, y) and E == E0 + g[i]
        else:
            assert np.array_equal(x, x0) and E == E0


def test_tabu_ties_go_to_the_lowest_index(orc):
    """Reading S6: among equal move values the lowest index moves.  With Q
    diagonal and all Q_ii equal every free variable has the same gain, so the
    search moves 0, 1, 2, ... in turn (each stays tabu with c = n) and every
    move lowers the energy: x_min holds ones at the first alpha indices."""
    n = 7
    Q = np.diag([-5] * n).astype(np.int8)
    for alpha in range(1, n + 1):
        x, E, T, C = orc.tabu(Q, np.zeros(n, np.uint8), alpha, n)
        assert x.tolist() == [1] * alpha + [0] * (n - alpha), alpha
        assert E == -5 * alpha and T.tolist() == x.tolist()


def test_tabu_long_tenure_never_repeats_and_never_worsens(orc):
    Q = make_qubo(60, 0.3, 2)
    x0 = random_solutions(60, 1, 2)[0]
    x, E, T, C = orc.tabu(Q, x0, 25, 26)
    assert T.max() == 1 and T.sum() == 25
    assert E <= orc.energy(Q, x0)


def test_tabu_result_is_no_better_than_the_optimum(orc):
    Q = make_qubo(14, 1.0, 6)
    opt, _ = brute_min(Q)
    for x0 in random_solutions(14, 4, 6):
        x, E, T, C = orc.tabu(Q, x0, 70, 2)
        assert E >= opt and E == orc.energy(Q, x)


# ----------------------------------------------------------------------------- Eq. 6-8, Algorithm 3
def test_control_parameters_hand_worked_example(orc):
    g = _gold("control3_worked.json")
    Q = np.array(g["Q"], dtype=np.int8)
    eta = orc.eta(Q)
    assert eta.tolist() == g["eta"]
    eh = orc.eta_hat(eta)
    assert eh.tolist() == g["eta_hat"]
    gam = orc.gamma(np.array(g["S"], np.uint8))
    assert gam.tolist() == g["gamma"]
    dl = orc.delta(np.array(g["T"], np.int32))
    assert dl.tolist() == g["delta"]
    A = orc.aggregate(eh, gam, dl, g["w"])
    assert A.tolist() == g["A"]
    assert orc.rank(A).tolist() == g["rank"]
    fc = g["floor_case"]
    assert orc.aggregate(fc["eta_hat"], fc["gamma"], fc["delta"], g["w"]).tolist() == fc["A"]


def test_gamma_takes_the_closed_form_values_for_z4(orc):
    # column sums 0..4 over z = 4 solutions give gamma = 1 - |s - 2| / 2
    S = np.array([[0, 1, 1, 1, 1], [0, 0, 1, 1, 1], [0, 0, 0, 1, 1], [0, 0, 0, 0, 1]], np.uint8)
    assert orc.gamma(S).tolist() == [0, 32768, 65536, 32768, 0]
    S3 = np.array([[1, 0], [0, 0], [1, 1]], np.uint8)          # z = 3: sums 2, 1
    assert orc.gamma(S3).tolist() == [(3 - 1) * 65536 // 3, (3 - 1) * 65536 // 3]


def test_delta_closed_forms(orc):
    assert orc.delta(np.array([0, 1, 2, 4], np.int32)).tolist() == [65536, 49152, 32768, 0]
    assert orc.delta(np.zeros(5, np.int32)).tolist() == [0] * 5
    assert orc.delta(np.array([3, 3], np.int32)).tolist() == [0, 0]


def test_eta_is_symmetric_column_abs_sum(orc):
    Q = make_qubo(40, 0.4, 3)
    e = orc.eta(Q)
    assert np.array_equal(e, np.abs(Q.astype(np.int64)).sum(axis=1))  # Q symmetric: rows = columns
    eh = orc.eta_hat(e)
    assert eh.max() == 65536 and eh.min() >= 0
    assert orc.eta_hat(np.zeros(4, np.int64)).tolist() == [0, 0, 0, 0]


# ----------------------------------------------------------------------------- selection
def _check_selection(A, sizes, idx):
    n = A.shape[0]
    M = int(sum(sizes))
    assert len(idx) == M and len(set(idx.tolist())) == M
    sel = np.zeros(n, bool)
    sel[idx] = True
    # every selected variable outranks every unselected one, index breaking ties
    for i in np.nonzero(sel)[0]:
        for j in np.nonzero(~sel)[0]:
            assert A[i] > A[j] or (A[i] == A[j] and i < j)
    off = 0
    groups = []
    for m in sizes:
        gk = idx[off:off + m]
        assert np.all(np.diff(gk) > 0)
        groups.append(gk)
        off += m
    for a in range(len(groups) - 1):
        for i in groups[a]:
            for j in groups[a + 1]:
                assert A[i] > A[j] or (A[i] == A[j] and i < j)


def test_selection_properties(orc):
    rng = np.random.default_rng(0)
    for n, sizes in [(50, [10]), (64, [7, 3, 12]), (40, [40]), (33, [1, 1, 1])]:
        for ties in (False, True):
            A = rng.integers(-5, 5, n) if ties else rng.permutation(n) * 3 - 20
            A = A.astype(np.int32)
            idx = orc.select(A, np.array(sizes, np.int32))
            _check_selection(A, sizes, idx)


def test_subqubo_sizes(orc):
    s = orc.subqubo_sizes(16, 64, 64, 5, 0, 0)
    assert s.tolist() == [64] * 16
    allsz = np.concatenate([orc.subqubo_sizes(16, 32, 256, 7, p, t) for p in range(8) for t in range(8)])
    assert allsz.min() >= 32 and allsz.max() <= 256
    assert abs(allsz.mean() - 144) < 12
    assert not np.array_equal(orc.subqubo_sizes(16, 32, 256, 7, 0, 0), orc.subqubo_sizes(16, 32, 256, 7, 0, 1))


# ----------------------------------------------------------------------------- Eq. 4
@pytest.mark.parametrize("n,m,seed", [(30, 6, 1), (25, 10, 2), (40, 8, 3)])
def test_subqubo_energy_differences_equal_full_energy_differences(orc, n, m, seed):
    """Eq. 4: for every pair of assignments y, y' of the subQUBO variables,
    f_sub(y) - f_sub(y') = f(x with S := y) - f(x with S := y')."""
    Q = make_qubo(n, 0.7, seed)
    x = random_solutions(n, 1, seed)[0]
    S = random_subsets(n, [m], seed)
    Qs, b = orc.subqubo(Q, x, S)
    Y = np.array(list(itertools.product([0, 1], repeat=m)), dtype=np.uint8)
    fsub = np.array([orc.subqubo_energy(Qs, y) for y in Y])
    full = []
    for y in Y:
        z = x.copy()
        z[S] = y
        full.append(orc.energy(Q, z))
    full = np.array(full)
    assert np.all((fsub - full) == (fsub[0] - full[0]))


def test_subqubo_local_gain_equals_global_gain(orc):
    Q = make_qubo(80, 0.3, 4)
    x = random_solutions(80, 1, 4)[0]
    S = random_subsets(80, [16], 4)
    Qs, b = orc.subqubo(Q, x, S)
    g = orc.gains(Q, x)
    xs = x[S]
    for a in range(16):
        y = xs.copy()
        y[a] ^= 1
        assert orc.subqubo_energy(Qs, y) - orc.subqubo_energy(Qs, xs) == g[S[a]]


# ----------------------------------------------------------------------------- anneal
def _sub(orc, n=60, m=12, seed=1):
    Q = make_qubo(n, 1.0, seed)
    x = random_solutions(n, 1, seed)[0]
    S = random_subsets(n, [m], seed)
    Qs, _ = orc.subqubo(Q, x, S)
    return Qs, x[S]


def test_anneal_infinite_temperature_accepts_every_attempt(orc):
    Qs, xs = _sub(orc)
    nlog = orc.nlog_table()
    beta = np.zeros(3, np.uint32)
    x1, dE, acc = orc.anneal(Qs, xs, beta[:1], nlog, 9, 0, 0)
    assert acc == 12 and np.array_equal(x1, 1 - xs)
    x3, dE3, acc3 = orc.anneal(Qs, xs, beta, nlog, 9, 0, 0)
    assert acc3 == 36 and np.array_equal(x3, 1 - xs)
    assert dE3 == orc.subqubo_energy(Qs, x3) - orc.subqubo_energy(Qs, xs)


def test_anneal_zero_temperature_is_greedy_descent_to_a_local_minimum(orc):
    Qs, xs = _sub(orc, seed=3)
    nlog = orc.nlog_table()
    beta = np.full(50, 2 ** 32 - 1, np.uint32)
    x1, dE, acc = orc.anneal(Qs, xs, beta, nlog, 1, 0, 0)
    E0 = orc.subqubo_energy(Qs, xs)
    E1 = orc.subqubo_energy(Qs, x1)
    assert dE == E1 - E0 and E1 <= E0
    for a in range(len(xs)):
        y = x1.copy()
        y[a] ^= 1
        assert orc.subqubo_energy(Qs, y) >= E1


def test_anneal_energy_change_is_exact(orc):
    for seed in range(4):
        Qs, xs = _sub(orc, n=100, m=20, seed=seed)
        beta = orc.beta_table(64, 400.0, 1.0)
        x1, dE, acc = orc.anneal(Qs, xs, beta, orc.nlog_table(), seed, 3, 7)
        assert dE == orc.subqubo_energy(Qs, x1) - orc.subqubo_energy(Qs, xs)
        assert 0 < acc < 64 * 20


def test_anneal_slow_schedule_finds_the_subqubo_optimum(orc):
    """m = 10: a slow cosine schedule reaches the exhaustive minimum of the
    subQUBO, and never goes below it."""
    for seed in range(3):
        Qs, xs = _sub(orc, n=50, m=10, seed=seed + 10)
        Y = np.array(list(itertools.product([0, 1], repeat=10)), dtype=np.uint8)
        opt = min(orc.subqubo_energy(Qs, y) for y in Y)
        beta = orc.beta_table(400, 600.0, 0.5)
        x1, dE, acc = orc.anneal(Qs, xs, beta, orc.nlog_table(), 100 + seed, 0, 0)
        assert orc.subqubo_energy(Qs, x1) == opt


@pytest.mark.parametrize("m,seed", [(1, 0), (4, 1), (7, 2), (10, 3)])
def test_exact_subqubo_is_the_full_energy_minimum(orc, m, seed):
    """The exact Ising machine (all 2^m assignments of the subQUBO) against an
    independent enumeration of the whole energy (Eq. 1) with the other
    variables fixed; ties to the smallest assignment sum_a y_a 2^a."""
    n = 30
    Q = make_qubo(n, 0.7, seed)
    x = random_solutions(n, 1, seed)[0]
    S = np.sort(np.random.default_rng(seed).choice(n, m, replace=False)).astype(np.int32)
    Qs, _ = orc.subqubo(Q, x, S)
    y, dE = orc.exact_subqubo(Qs, x[S])
    best = None
    for v in range(1 << m):
        xv = x.copy()
        xv[S] = [(v >> a) & 1 for a in range(m)]
        e = full_energy(Q, xv)
        if best is None or e < best[0]:
            best = (e, v)
    assert [int(b) for b in y] == [(best[1] >> a) & 1 for a in range(m)]
    assert dE == best[0] - full_energy(Q, x)


def test_exact_subqubo_ties_take_the_smallest_assignment(orc):
    Qs = np.zeros((3, 3), np.int32)           # f = 0 everywhere: the answer is y = 0
    y, dE = orc.exact_subqubo(Qs, np.array([1, 0, 1], np.uint8))
    assert y.tolist() == [0, 0, 0] and dE == 0
    Qs = np.diag([-5, 0, -5]).astype(np.int32)  # y_1 is free: the smaller choice y_1 = 0
    y, dE = orc.exact_subqubo(Qs, np.array([0, 1, 0], np.uint8))
    assert y.tolist() == [1, 0, 1] and dE == -10


def test_anneal_acceptance_frequency_matches_the_table(orc):
    """One variable (m = 1) with a fixed positive gain: the accepted fraction
    over many independent attempts is the table's probability."""
    l = 40
    Qs = np.array([[l]], np.int32)        # x = 0 -> gain l; x = 1 -> gain -l (always accepted back)
    nlog = orc.nlog_table()
    T = 30.0
    beta = np.full(1, round(2 ** 24 / T), np.uint32)
    acc = 0
    N = 20000
    for it in range(N):
        _, _, a = orc.anneal(Qs, np.zeros(1, np.uint8), beta, nlog, 5, 0, it)
        acc += a
    p = (l * int(beta[0]) < nlog.astype(np.int64)).sum() / 4096
    assert abs(acc / N - p) < 4 * math.sqrt(p * (1 - p) / N) + 1e-3
    assert abs(p - math.exp(-l / T)) < 2e-3


def test_anneal_is_deterministic_in_seed_slot_and_iteration(orc):
    Qs, xs = _sub(orc, seed=2)
    beta = orc.beta_table(32, 200.0, 1.0)
    nlog = orc.nlog_table()
    a = orc.anneal(Qs, xs, beta, nlog, 1, 2, 3)
    assert a[0].tolist() == orc.anneal(Qs, xs, beta, nlog, 1, 2, 3)[0].tolist()
    others = [orc.anneal(Qs, xs, beta, nlog, *k)[2] for k in [(2, 2, 3), (1, 3, 3), (1, 2, 4)]]
    assert any(o != a[2] for o in others)


# ----------------------------------------------------------------------------- mutation
def test_mutation_only_touches_the_top_L_outside_S_prime(orc):
    rng = np.random.default_rng(5)
    n = 200
    A = rng.integers(-1000, 5000, n).astype(np.int32)
    sel = np.zeros(n, np.uint8)
    sel[orc.select(A, np.array([30], np.int32))] = 1
    order = [i for i in orc.rank(A) if not sel[i]]
    for L in (0, 1, 17, 170):
        x0 = random_solutions(n, 1, L)[0]
        total = 0
        for it in range(20):
            x1, f = orc.mutate(A, sel, L, 3, 0, it, x0)
            changed = set(np.nonzero(x1 != x0)[0].tolist())
            assert changed <= set(order[:L]) and len(changed) == f
            total += f
        if L == 0:
            assert total == 0


def test_mutation_flip_frequency_follows_normalised_A(orc):
    n = 64
    A = np.linspace(0, 63 * 1000, n).astype(np.int32)       # A_min at index 0, A_max at 63
    sel = np.zeros(n, np.uint8)
    counts = np.zeros(n)
    N = 3000
    for it in range(N):
        x1, _ = orc.mutate(A, sel, n, 11, 2, it, np.zeros(n, np.uint8))
        counts += x1
    freq = counts / N
    P = (A - A.min()) / (A.max() - A.min())
    assert counts[0] == 0                       # P = 0 for the minimum
    assert np.all(np.abs(freq - P) < 4 * np.sqrt(P * (1 - P) / N) + 3e-3)
    # constant A: probability 1/2
    x1s = [orc.mutate(np.full(n, 7, np.int32), sel, n, 11, 2, it, np.zeros(n, np.uint8))[0] for it in range(200)]
    assert abs(np.mean(x1s) - 0.5) < 0.02


# ----------------------------------------------------------------------------- Algorithm 2
@pytest.mark.parametrize("n,seed", [(12, 0), (16, 1), (18, 2)])
def test_run_reaches_the_brute_force_optimum(orc, n, seed):
    Q = make_qubo(n, 1.0, seed)
    opt, argmins = brute_min(Q)
    prm = orc.default_params(n, m=4, max_iters=30, patience=0, sweeps=64, T_max=300.0)
    r = orc.run(Q, prm, 1000 + seed)
    assert r["best_E"] == opt
    assert orc.energy(Q, r["best_x"]) == r["best_E"]
    assert any(np.array_equal(r["best_x"], a) for a in argmins)


def test_run_trace_is_consistent(orc):
    n = 64
    Q = make_qubo(n, 1.0, 3)
    prm = orc.default_params(n, m=16, z=8, max_iters=12, patience=0, sweeps=32, T_max=2000.0, alpha=40)
    r = orc.run(Q, prm, 77)
    tr = r["trace"]
    z = 8
    assert tr.shape == (12, 3 * z + 1)
    best = tr[:, 3 * z]
    assert np.all(np.diff(best) <= 0)
    assert best[-1] == r["best_E"] <= r["init_best_E"]
    assert best[0] <= min(tr[0, :3 * z].min(), r["init_best_E"])
    assert np.array_equal(orc.energy_batch(Q, r["S"]), tr[-1, 2 * z:3 * z])
    # the Tabu search never returns a worse solution than it started from
    for t in range(1, 12):
        assert np.all(tr[t, :z] <= tr[t - 1, 2 * z:3 * z])
    assert np.all(tr[0, :z] <= r["init_E"])


def test_run_patience_stops_and_is_deterministic(orc):
    n = 24
    Q = make_qubo(n, 1.0, 9)
    prm = orc.default_params(n, m=8, max_iters=500, patience=3, sweeps=16)
    r1 = orc.run(Q, prm, 5)
    r2 = orc.run(Q, prm, 5)
    assert r1["iters"] < 500
    assert r1["best_E"] == r2["best_E"] and np.array_equal(r1["trace"], r2["trace"])
    tr = r1["trace"][:, -1]
    # the last `patience` iterations did not improve on what came before them
    assert np.all(tr[-3:] == tr[-4]) if len(tr) >= 4 else True


def test_run_is_the_chain_of_its_steps_from_what_a_checkpoint_holds(orc):
    """Resuming a run needs only the solutions, the best solution and energy,
    the hit counts, the stale count, the seed and t: Algorithm 2 run whole
    equals its initial pass followed by single steps that receive exactly
    those quantities (and the chain stops by patience where the run does)."""
    n, seed = 90, 11
    Q = make_qubo(n, 0.6, 21)
    for patience, iters in ((0, 10), (2, 200)):
        prm = orc.default_params(n, z=4, K=2, m_min=6, m_max=12, m_init=12, max_iters=iters, patience=patience,
                                 sweeps=16, T_max=300.0, alpha=n)
        r = orc.run(Q, prm, seed)
        S = orc.init_solutions(n, prm.z, seed)
        S, E = orc.initial_pass(Q, prm, seed, S)
        b = int(np.argmin(E))
        best_E, best_x = int(E[b]), S[b].copy()
        assert best_E == r["init_best_E"]
        H = np.zeros((prm.z, n), np.int32)
        stale, rows, t = 0, [], 0
        while t < iters and (patience <= 0 or stale < patience):
            st = orc.step(Q, prm, seed, t, S, best_E, best_x, H=H)
            stale = 0 if st["best_E"] < best_E else stale + 1
            S, best_E, best_x, H = st["S"], st["best_E"], st["best_x"], st["H"]
            rows.append(np.concatenate([st["trace3"], [best_E]]))
            t += 1
        assert t == r["iters"] and (patience == 0 or t < iters)
        assert np.array_equal(np.stack(rows), r["trace"])
        assert np.array_equal(S, r["S"]) and best_E == r["best_E"] and np.array_equal(best_x, r["best_x"])


def test_run_batched_uneven_subqubos(orc):
    n = 200
    Q = make_qubo(n, 0.5, 4)
    prm = orc.default_params(n, z=3, K=4, m_min=8, m_max=24, m_init=20, max_iters=4, patience=0,
                             sweeps=16, alpha=100, T_max=3000.0)
    r = orc.run(Q, prm, 3)
    assert r["iters"] == 4 and r["best_E"] == orc.energy(Q, r["best_x"])
    assert np.all(np.diff(r["trace"][:, -1]) <= 0)


# ----------------------------------------------------------------------------- ablations (Section 4, Fig. 23)
def _abl_setup(orc, ablation, n=60, z=4, seed=5):
    Q = make_qubo(n, 0.5, seed)
    prm = orc.default_params(n, z=z, K=2, m_min=6, m_max=9, m_init=10, alpha=2 * n, c=3, sweeps=16, T_max=80.0,
                             mut_mode=0, max_iters=3)
    prm.ablation = ablation
    S = random_solutions(n, z, seed + 1)
    return Q, prm, S


def test_no_im_ablation_is_tabu_then_mutation(orc):
    """No_IM: the Ising-machine phase changes nothing and selects nothing; the
    step is the Tabu search followed by the mutation over all variables."""
    Q, prm, S = _abl_setup(orc, 1)
    t, seed, n, z = 0, 11, Q.shape[0], prm.z
    r = orc.step(Q, prm, seed, t, S, H=np.zeros(S.shape, np.int32))
    assert np.array_equal(r["trace3"][z:2 * z], r["trace3"][:z]) and not r["H"].any()
    eh = orc.eta_hat(orc.eta(Q))
    X = np.stack([orc.tabu(Q, S[p], prm.alpha, prm.c)[0] for p in range(z)])
    gam = orc.gamma(X)
    L = int(np.floor(n * orc.mutation_rate(t)))
    for p in range(z):
        _, _, T, _ = orc.tabu(Q, S[p], prm.alpha, prm.c)
        A = orc.aggregate(eh, gam, orc.delta(T))
        want, _ = orc.mutate(A, np.zeros(n, np.uint8), L, seed, p, t, X[p])
        assert np.array_equal(r["S"][p], want)


def test_no_sm_ablation_ranks_at_random_and_flips_with_probability_half(orc):
    """No_SM: S' and the mutation candidates come from the ranking of the
    Philox keys (ctr (j/4, 7 << 24, p, t)) >> 1 instead of A, and every
    candidate flips iff its mutation word is below 2^31."""
    Q, prm, S = _abl_setup(orc, 2, n=80, seed=9)
    t, seed, n, z = 1, 21, Q.shape[0], prm.z
    r = orc.step(Q, prm, seed, t, S, H=np.zeros(S.shape, np.int32))
    key = np.array([seed & 0xffffffff, seed >> 32], np.uint32)
    for p in range(z):
        rk = np.array([orc.philox([j // 4, 7 << 24, p, t], key)[j % 4] >> 1 for j in range(n)], np.int64)
        sizes = orc.subqubo_sizes(prm.K, prm.m_min, prm.m_max, seed, p, t)
        sel = np.sort(orc.select(rk.astype(np.int32), sizes))
        assert np.flatnonzero(r["H"][p]).tolist() == sel.tolist()
    # mutation: the first L candidates outside S' in the random order, each
    # flipped iff its word is below 2^31 (the state before the mutation comes
    # from the same step with a zero mutation rate)
    prm0 = orc.Params.from_buffer_copy(prm)
    prm0.mut_mode, prm0.mut_rate = 1, 0.0
    r0 = orc.step(Q, prm0, seed, t, S, H=np.zeros(S.shape, np.int32))
    flipped_any = False
    for p in range(z):
        rk = np.array([orc.philox([j // 4, 7 << 24, p, t], key)[j % 4] >> 1 for j in range(n)], np.int64)
        sel = set(np.flatnonzero(r["H"][p]).tolist())
        L = int(np.floor((n - len(sel)) * orc.mutation_rate(t)))
        cands = [j for j in orc.rank(rk.astype(np.int32)).tolist() if j not in sel][:L]
        want = r0["S"][p].copy()
        for j in cands:
            if orc.philox([j // 4, 3 << 24, p, t], key)[j % 4] < 2 ** 31:
                want[j] ^= 1
        assert np.array_equal(r["S"][p], want)
        flipped_any |= bool((want != r0["S"][p]).any())
    assert flipped_any


# ----------------------------------------------------------------------------- aspiration (reading S4)
def _replay_aspiration(Q, x0, alpha, c):
    """The aspiration rule executed with full energies (Eq. 1 from scratch):
    the lowest E(x with x_k flipped) among the free variables and the tabu ones
    that beat the best visited; if there are none, among all (reading S6);
    ties to the lowest index.  Returns (moves, best E, best x, fallbacks, aspirated)."""
    n = Q.shape[0]
    x = x0.copy()
    Ebest, xbest = full_energy(Q, x), x.copy()
    C = np.zeros(n, np.int64)
    moves, fallbacks, aspirated = [], 0, 0
    for _ in range(alpha):
        e = [full_energy(Q, np.where(np.arange(n) == k, 1 - x, x)) for k in range(n)]
        cand = [(e[k], k) for k in range(n) if C[k] <= 0 or e[k] < Ebest]
        if not cand:
            cand = [(e[k], k) for k in range(n)]
            fallbacks += 1
        ek, k = min(cand)
        aspirated += int(C[k] > 0)
        moves.append(k)
        x[k] ^= 1
        C[k] += c
        C[C > 0] -= 1
        if ek < Ebest:
            Ebest, xbest = ek, x.copy()
    return moves, Ebest, xbest, fallbacks, aspirated


def test_tabu_with_aspiration_follows_the_rule_by_full_energies(orc):
    fired = 0
    for seed in range(12):
        n = 6 + seed % 5
        Q = make_qubo(n, 1.0, 300 + seed)
        x0 = random_solutions(n, 1, seed)[0]
        alpha, c = 4 * n, n - 1
        xm, Em, T, Cm, mv = orc.tabu_asp(Q, x0, alpha, c)
        moves, Eb, xb, _, asp = _replay_aspiration(Q, x0, alpha, c)
        assert mv.tolist() == moves and Em == Eb and np.array_equal(xm, xb), seed
        fired += asp
    assert fired > 0


def test_tabu_with_aspiration_when_every_move_is_tabu(orc):
    """Tenure c = n: a variable moved while tabu keeps c more iterations of
    tabu memory, every move becomes tabu, and the search takes the unmasked
    arg-min (instances where this happens, found by a search over seeds)."""
    falls = 0
    for seed in (0, 6, 12, 14, 16, 18):
        n = 4 + seed % 5
        Q = make_qubo(n, 1.0, 1000 + seed)
        x0 = random_solutions(n, 1, seed)[0]
        xm, Em, T, Cm, mv = orc.tabu_asp(Q, x0, 8 * n, n)
        moves, Eb, xb, fb, _ = _replay_aspiration(Q, x0, 8 * n, n)
        assert mv.tolist() == moves and Em == Eb and np.array_equal(xm, xb), seed
        falls += fb
    assert falls > 0


def test_tabu_without_aspiration_is_algorithm_1(orc):
    Q = make_qubo(40, 0.5, 3)
    x0 = random_solutions(40, 1, 4)[0]
    a = orc.tabu(Q, x0, 200, 5)
    b = orc.tabu_asp(Q, x0, 200, 5, aspiration=False)
    assert np.array_equal(a[0], b[0]) and a[1] == b[1]
    assert np.array_equal(a[2], b[2]) and np.array_equal(a[3], b[3])


# ----------------------------------------------------------------------------- Gauss-Seidel multi-IM order
def _im_phase_by_pieces(orc, Q, prm, seed, t, S, gauss_seidel):
    """The Ising-machine phase of one step rebuilt from the pinned pieces:
    Tabu search, gamma / delta / A, the subQUBO sizes and groups, then each
    group's subQUBO (Eq. 4) annealed and written back -- built from the state
    before the call (Jacobi) or from the state the earlier groups left
    (Gauss-Seidel)."""
    n, z, K = Q.shape[0], prm.z, prm.K
    eh = orc.eta_hat(orc.eta(Q))
    tab = [orc.tabu(Q, S[p], prm.alpha, prm.c) for p in range(z)]
    X = np.stack([r[0] for r in tab])
    gam = orc.gamma(X)
    beta, nlog = orc.beta_table(prm.sweeps, prm.T_max, prm.T_min), orc.nlog_table()
    out = X.copy()
    for p in range(z):
        A = orc.aggregate(eh, gam, orc.delta(tab[p][2]))
        sizes = orc.subqubo_sizes(K, prm.m_min, prm.m_max, seed, p, t)
        idx = orc.select(A, sizes)
        pre, off = X[p].copy(), 0
        for k, m in enumerate(sizes):
            grp = idx[off:off + m]
            base = out[p] if gauss_seidel else pre
            Qs, _ = orc.subqubo(Q, base, grp)
            xs, _, _ = orc.anneal(Qs, base[grp], beta, nlog, seed, p * K + k, t)
            out[p, grp] = xs
            off += m
    return out


def test_gauss_seidel_order_of_the_subqubos(orc):
    """im_order 1: group k's subQUBO is built from the solution with groups
    0..k-1 already written back; im_order 0 builds every group from the
    solution before the call.  Both equal the step rebuilt from its pinned
    pieces (the mutation is switched off so the step ends with the IM phase),
    they differ on some solution, and with K = 1 they are the same step."""
    Q = make_qubo(70, 0.6, 17)
    n, z, seed, t = 70, 5, 23, 2
    # a short Tabu search leaves the solutions far from a local minimum, so the
    # Ising machine changes many variables and the two orders part
    prm = orc.default_params(n, z=z, K=4, m_min=5, m_max=12, m_init=10, alpha=5, c=3, sweeps=24,
                             T_max=120.0, mut_mode=1, mut_rate=0.0, max_iters=3)
    S = random_solutions(n, z, 31)
    res = {}
    for order in (0, 1):
        prm.im_order = order
        r = orc.step(Q, prm, seed, t, S)
        want = _im_phase_by_pieces(orc, Q, prm, seed, t, S, order == 1)
        assert np.array_equal(r["S"], want), order
        assert np.array_equal(r["E"], orc.energy_batch(Q, want))
        res[order] = r["S"]
    assert not np.array_equal(res[0], res[1])
    prm.K, prm.m_min, prm.m_max = 1, 12, 12
    prm.im_order = 0
    a = orc.step(Q, prm, seed, t, S)["S"]
    prm.im_order = 1
    assert np.array_equal(orc.step(Q, prm, seed, t, S)["S"], a)


def _initial_pass_by_pieces(orc, Q, prm, seed, S, G):
    """Call_IM_Solution_Set rebuilt from the pinned pieces: blocks of m_init
    consecutive variables, G at a time, each built from the solution before
    its group (G = 1: before the block itself)."""
    n, m = Q.shape[0], prm.m_init
    nb = n // m
    beta, nlog = orc.beta_table(prm.sweeps, prm.T_max, prm.T_min), orc.nlog_table()
    out = S.copy()
    for p in range(prm.z):
        x = out[p]
        for l0 in range(0, nb, G):
            pre = x.copy()
            for l in range(l0, min(l0 + G, nb)):
                grp = np.arange(l * m, (l + 1) * m, dtype=np.int32)
                Qs, _ = orc.subqubo(Q, pre, grp)
                xs, _, _ = orc.anneal(Qs, pre[grp], beta, nlog, seed, p, 0x80000000 | l)
                x[grp] = xs
    return out


def test_initial_pass_with_several_ising_machines(orc):
    """K > 1 IMs per solution (Jacobi order): Call_IM_Solution_Set solves K
    consecutive blocks at once, each from the solution before the group
    (reading S24); K = 1, or the Gauss-Seidel order, keeps one block at a
    time.  Both equal the pass rebuilt from its pieces, and they differ."""
    n, z, seed = 70, 3, 41
    Q = make_qubo(n, 0.6, 43)
    S = random_solutions(n, z, 44)
    prm = orc.default_params(n, z=z, K=3, m_min=4, m_max=8, m_init=8, sweeps=20, T_max=150.0)
    grouped, _ = orc.initial_pass(Q, prm, seed, S)
    assert np.array_equal(grouped, _initial_pass_by_pieces(orc, Q, prm, seed, S, 3))
    prm.im_order = 1
    seq, _ = orc.initial_pass(Q, prm, seed, S)
    assert np.array_equal(seq, _initial_pass_by_pieces(orc, Q, prm, seed, S, 1))
    prm.im_order, prm.K = 0, 1
    assert np.array_equal(orc.initial_pass(Q, prm, seed, S)[0], seq)
    assert not np.array_equal(grouped, seq)
