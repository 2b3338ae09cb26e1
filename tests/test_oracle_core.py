"""Pins of the CPU oracle's core arithmetic against what the paper and the
mathematics fix: Philox against an independent generator, Eq. 1 against
hand-worked values and the Ising form (Eq. 2-3), the 1-flip move value
against the closed-form energy difference, and the host tables against the
Metropolis closed form.  No GPU."""
import ctypes
import ctypes.util
import itertools
import json
import math
import os

import numpy as np
import pytest

from paper_2502_13947_gb300.instances import make_qubo, random_solutions

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _gold(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def _curand():
    for cand in ("/usr/local/cuda/lib64/libcurand.so", ctypes.util.find_library("curand")):
        if not cand:
            continue
        try:
            return ctypes.CDLL(cand)
        except OSError:
            pass
    return None


# ----------------------------------------------------------------------------- Philox
def test_philox_first_block_matches_curand_host_generator(orc):
    """cuRAND's host PHILOX4_32_10 generator, seeded with s and read from
    offset 0, emits the block at counter 0 with key (s_lo, s_hi).  It is an
    independent implementation of the SC'11 definition, called as a library."""
    cr = _curand()
    if cr is None:
        pytest.skip("libcurand not available")
    for seed in (0, 1, 0x123456789ABCDEF, 0xFFFFFFFFFFFFFFFF, 42 << 32, 7):
        gen = ctypes.c_void_p()
        assert cr.curandCreateGeneratorHost(ctypes.byref(gen), 161) == 0  # CURAND_RNG_PSEUDO_PHILOX4_32_10
        assert cr.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        out = (ctypes.c_uint32 * 4)()
        assert cr.curandGenerate(gen, out, ctypes.c_size_t(4)) == 0
        cr.curandDestroyGenerator(gen)
        mine = orc.philox([0, 0, 0, 0], [seed & 0xFFFFFFFF, seed >> 32])
        assert list(mine) == list(out), hex(seed)


def _curand_blocks(cr, seed, offset, count):
    gen = ctypes.c_void_p()
    assert cr.curandCreateGeneratorHost(ctypes.byref(gen), 161) == 0  # CURAND_RNG_PSEUDO_PHILOX4_32_10
    try:
        assert cr.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        assert cr.curandSetGeneratorOffset(gen, ctypes.c_ulonglong(offset)) == 0
        out = (ctypes.c_uint32 * (4 * count))()
        assert cr.curandGenerate(gen, out, ctypes.c_size_t(4 * count)) == 0
    finally:
        cr.curandDestroyGenerator(gen)
    return [list(out[4 * b:4 * b + 4]) for b in range(count)]


def test_philox_counter_words_0_to_2_match_curand_host_generator(orc):
    """Counter words 0, 1 and 2 placed as the SC'11 definition places them.
    cuRAND's host generator (default ordering) emits, as its output block
    q = s * 65536 + t, the block at counter (s mod 2^32, s div 2^32, t, 0):
    65536 subsequences in word 2, the position within one in words 0-1.
    Reading it at offsets 4q therefore pins word 0 over its whole range,
    word 1 through positions beyond 2^32, and word 2; word 3 is the one slot
    left, and the next test shows that it changes the block."""
    cr = _curand()
    if cr is None:
        pytest.skip("libcurand not available")
    for seed in (0x123456789ABCDEF, 7, 0xFFFFFFFFFFFFFFFF):
        key = [seed & 0xFFFFFFFF, seed >> 32]
        for s, t in ((0, 1), (1, 0), (12345, 40000), (1 << 32, 0), (3 * (1 << 32) + 5, 7),
                     ((1 << 40) + 0xDEADBEEF, 65535), (0xFFFFFFFF, 65535)):
            got = _curand_blocks(cr, seed, 4 * (s * 65536 + t), 2)
            for b in range(2):
                q = s * 65536 + t + b
                ss, tt = q // 65536, q % 65536
                mine = orc.philox([ss & 0xFFFFFFFF, ss >> 32, tt, 0], key)
                assert list(mine) == got[b], (hex(seed), s, t, b)


def test_philox_counter_words_all_matter_and_output_is_uniform(orc):
    base = orc.philox([5, 6, 7, 8], [9, 10])
    for w in range(4):
        c = [5, 6, 7, 8]
        c[w] ^= 1
        assert list(orc.philox(c, [9, 10])) != list(base)
    for w in range(2):
        k = [9, 10]
        k[w] ^= 1
        assert list(orc.philox([5, 6, 7, 8], k)) != list(base)
    words = np.concatenate([orc.philox([i, 3, 2, 1], [77, 88]) for i in range(4000)])
    bits = np.unpackbits(words.view(np.uint8))
    assert abs(bits.mean() - 0.5) < 0.005
    hist = np.bincount(words >> 28, minlength=16)
    chi2 = ((hist - words.size / 16) ** 2 / (words.size / 16)).sum()
    assert chi2 < 40.0  # 15 d.o.f., p ~ 5e-4


# ----------------------------------------------------------------------------- Eq. 1
def test_energy_hand_worked_example(orc):
    g = _gold("qubo3_worked.json")
    Q = np.array(g["Q"], dtype=np.int8)
    for bits, e in g["energies"].items():
        x = np.array([int(b) for b in bits], dtype=np.uint8)
        assert orc.energy(Q, x) == e
    assert orc.gains(Q, np.zeros(3, np.uint8)).tolist() == [2, -4, 1]


def test_energy_closed_forms(orc):
    Q = make_qubo(37, 1.0, 11)
    n = Q.shape[0]
    assert orc.energy(Q, np.zeros(n, np.uint8)) == 0
    for i in range(n):
        e = np.zeros(n, np.uint8)
        e[i] = 1
        assert orc.energy(Q, e) == Q[i, i]
    for i, j in [(0, 1), (3, 20), (36, 5)]:
        e = np.zeros(n, np.uint8)
        e[[i, j]] = 1
        assert orc.energy(Q, e) == int(Q[i, i]) + int(Q[j, j]) + 2 * int(Q[i, j])


def test_energy_equals_ising_form(orc):
    """Eq. 2-3: with s = 2x - 1, x^T Q x = (s^T Q s + 2 * 1^T Q s + 1^T Q 1) / 4."""
    Q = make_qubo(50, 0.3, 5)
    Qi = Q.astype(np.int64)
    one = np.ones(50, np.int64)
    for x in random_solutions(50, 20, 3):
        s = 2 * x.astype(np.int64) - 1
        ising = (s @ Qi @ s + 2 * one @ Qi @ s + one @ Qi @ one)
        assert ising % 4 == 0
        assert orc.energy(Q, x) == ising // 4


def test_gain_is_single_flip_energy_difference(orc):
    for n, d, seed in [(23, 1.0, 1), (40, 0.2, 2), (64, 1.0, 3)]:
        Q = make_qubo(n, d, seed)
        for x in random_solutions(n, 4, seed):
            g = orc.gains(Q, x)
            E = orc.energy(Q, x)
            for i in range(n):
                y = x.copy()
                y[i] ^= 1
                assert g[i] == orc.energy(Q, y) - E


def test_energy_batch_matches_single(orc):
    Q = make_qubo(31, 0.5, 9)
    X = random_solutions(31, 6, 1)
    assert orc.energy_batch(Q, X).tolist() == [orc.energy(Q, x) for x in X]


# ----------------------------------------------------------------------------- tables
def test_mutation_rate_closed_forms(orc):
    g = _gold("mutation_rate.json")
    for t, expr in g["values"].items():
        want = eval(expr, {"__builtins__": {}})
        got = orc.mutation_rate(int(t))
        assert abs(got - want) <= 1e-15, (t, got, want)
    assert orc.mutation_rate(15) == 0.0


def test_beta_schedule_endpoints_and_shape(orc):
    K, Tmax, Tmin = 257, 400.0, 2.0
    b = orc.beta_table(K, Tmax, Tmin)
    assert b[0] == round(2 ** 24 / Tmax)
    assert b[-1] == round(2 ** 24 / Tmin)
    assert b[128] == round(2 ** 24 / ((Tmax + Tmin) / 2))  # cos(pi/2) = 0 at the midpoint
    assert np.all(np.diff(b.astype(np.int64)) >= 0)       # temperature falls monotonically
    assert orc.beta_table(1, Tmax, Tmin).tolist() == [round(2 ** 24 / Tmin)]
    assert orc.beta_table(4, 1e12, 1e-12).tolist()[-1] == 2 ** 32 - 1  # saturates


def test_nlog_table_gives_metropolis_probability(orc):
    """Accept iff l * BETA < NLOG[u >> 20] with u uniform: the fraction of the
    4096 table entries above l * BETA must be exp(-l / T) within one table step."""
    t = orc.nlog_table().astype(np.int64)
    assert t.shape == (4096,)
    assert np.all(np.diff(t) < 0)
    for T in (3.0, 50.0, 1000.0):
        beta = round(2 ** 24 / T)
        for l in (1, 2, 5, 10, 30, 100, 500, 3000):
            p = (l * beta < t).sum() / 4096.0
            assert abs(p - math.exp(-l * beta / 2 ** 24)) <= 1.0 / 4096 + 1e-9, (T, l)


# ----------------------------------------------------------------------------- init
def test_initial_solutions_are_balanced_and_seeded(orc):
    S = orc.init_solutions(1000, 16, 1234)
    assert S.shape == (16, 1000) and set(np.unique(S)) <= {0, 1}
    assert abs(S.mean() - 0.5) < 0.02
    assert not np.array_equal(S[0], S[1])
    assert np.array_equal(S, orc.init_solutions(1000, 16, 1234))
    assert not np.array_equal(S, orc.init_solutions(1000, 16, 1235))
    # row p is independent of how many rows are drawn
    assert np.array_equal(orc.init_solutions(1000, 3, 1234), S[:3])


# ----------------------------------------------------------------------------- brute force
def all_energies(Q):
    n = Q.shape[0]
    X = np.array(list(itertools.product([0, 1], repeat=n)), dtype=np.int64)
    Qi = Q.astype(np.int64)
    return X, np.einsum("ki,ij,kj->k", X, Qi, X)


def test_brute_force_agrees_with_oracle_energy(orc):
    Q = make_qubo(10, 1.0, 4)
    X, E = all_energies(Q)
    got = orc.energy_batch(Q, X.astype(np.uint8))
    assert np.array_equal(got, E)
