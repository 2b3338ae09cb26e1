"""GPU parity: every step of the CUDA path, called through the C ABI, equals
the CPU oracle bit for bit on the same seeded inputs (integer, byte and index
results are exact by construction, so the bar is equality)."""
import numpy as np
import pytest

from paper_2502_13947_gb300 import build as B
from paper_2502_13947_gb300 import icd2s as I
from paper_2502_13947_gb300.instances import make_qubo, random_solutions, random_subsets

from .gpu_util import dev, lib_params, orc_params, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    torch_cuda()
    B.build()
    return I.lib()


class Problem:
    def __init__(self, n, density, seed, R=None, state_seed=11):
        self.n = n
        self.Q = make_qubo(n, density, seed)
        self.q = I.icd2s_qubo_create(self.Q)
        self.st = None
        if R:
            self.st = I.icd2s_state_create(self.q, R, state_seed)
            self.R = R
            self.seed = state_seed

    def load(self, X):
        I.icd2s_state_load(self.st, X)

    def state(self):
        return I.icd2s_get_state(self.st, self.R, self.n)

    def close(self):
        if self.st:
            I.icd2s_state_destroy(self.st)
        I.icd2s_qubo_destroy(self.q)


# ----------------------------------------------------------------------------- Eq. 1
@pytest.mark.parametrize("n,count,density", [(1, 1, 1.0), (64, 3, 1.0), (129, 5, 0.5), (300, 70, 0.3),
                                             (2500, 9, 0.1), (4097, 2, 1.0)])
def test_energy(L, orc, n, count, density):
    torch = torch_cuda()
    P = Problem(n, density, n + count)
    X = random_solutions(n, count, 3)
    E = torch.zeros(count, dtype=torch.int64, device="cuda")
    Xd = dev(X)
    I.icd2s_energy(P.q, Xd.data_ptr(), count, E.data_ptr())
    assert np.array_equal(E.cpu().numpy(), orc.energy_batch(P.Q, X))
    P.close()


def test_asymmetric_q_is_rejected(L):
    Q = make_qubo(40, 1.0, 1)
    Q[3, 7] = np.int8(Q[7, 3] + 1 if Q[7, 3] < 100 else Q[7, 3] - 1)
    with pytest.raises(I.ICD2SError) as e:
        I.icd2s_qubo_create(Q)
    assert e.value.code == I.ERR_ASYMMETRIC


# ----------------------------------------------------------------------------- init
@pytest.mark.parametrize("n,R", [(64, 1), (300, 7), (1000, 33)])
def test_initial_solutions_gains_and_energies(L, orc, n, R):
    P = Problem(n, 1.0, 5, R=R, state_seed=0xABCDEF0123)
    x, g, E = P.state()
    assert np.array_equal(x, orc.init_solutions(n, R, 0xABCDEF0123))
    for p in range(R):
        assert np.array_equal(g[p], orc.gains(P.Q, x[p]))
    assert np.array_equal(E, orc.energy_batch(P.Q, x))
    P.close()


# ----------------------------------------------------------------------------- Algorithm 1
@pytest.mark.parametrize("n,R,alpha,c,density", [
    (64, 4, 320, 2, 1.0),        # one warp
    (300, 3, 900, 3, 0.5),       # ragged n
    (2500, 2, 2000, 16, 0.1),    # 1 group of 4 per thread
    (5000, 2, 800, 33, 0.5),     # 2 groups per thread
    (10000, 1, 300, 66, 0.5),    # 3 groups per thread
    (13001, 1, 150, 86, 0.5),    # 4 groups per thread, ragged
    (50, 2, 0, 2, 1.0),          # alpha = 0: nothing moves
    (40, 2, 200, 40, 1.0),       # c = n
])
def test_tabu(L, orc, n, R, alpha, c, density):
    P = Problem(n, density, n, R=R)
    X0 = random_solutions(n, R, n + alpha)
    P.load(X0)
    I.icd2s_tabu(P.st, alpha, c)
    x, g, E = P.state()
    T, Cm = I.icd2s_get_tabu(P.st, R, n)
    for p in range(R):
        xo, Eo, To, Co = orc.tabu(P.Q, X0[p], alpha, c)
        assert np.array_equal(x[p], xo), p
        assert E[p] == Eo
        assert np.array_equal(T[p], To) and np.array_equal(Cm[p], Co)
        assert np.array_equal(g[p], orc.gains(P.Q, xo))
    P.close()


@pytest.mark.parametrize("n,R,alpha,c,variant", [(40, 3, 160, 39, -1), (300, 4, 900, 60, -1), (300, 2, 900, 60, 4),
                                                 (2500, 2, 5000, 16, -1), (5000, 2, 4000, 33, -1),
                                                 (5000, 2, 4000, 33, 3)])
def test_tabu_with_aspiration(L, orc, n, R, alpha, c, variant):
    """The aspiration criterion (reading S4) in several kernel shapes; long
    tenures make tabu moves that beat the best visited admissible."""
    P = Problem(n, 0.5, n + 1, R=R)
    X0 = random_solutions(n, R, n + c)
    P.load(X0)
    if variant >= 0:
        I.icd2s_set_tuning(P.st, tabu_variant=variant)
    I.icd2s_tabu_aspiration(P.st, alpha, c)
    x, g, E = P.state()
    T, Cm = I.icd2s_get_tabu(P.st, R, n)
    for p in range(R):
        xo, Eo, To, Co, _ = orc.tabu_asp(P.Q, X0[p], alpha, c)
        assert np.array_equal(x[p], xo), p
        assert E[p] == Eo
        assert np.array_equal(T[p], To) and np.array_equal(Cm[p], Co)
        assert np.array_equal(g[p], orc.gains(P.Q, xo))
    P.close()


def test_tabu_with_aspiration_when_every_move_is_tabu(L, orc):
    """Tenure c = n: every move becomes tabu and the kernel takes the
    unmasked arg-min like the oracle (instances where this happens)."""
    for seed in (0, 6, 12, 14, 16, 18):
        n = 4 + seed % 5
        P = Problem(n, 1.0, 1000 + seed, R=1)
        X0 = random_solutions(n, 1, seed)
        P.load(X0)
        I.icd2s_tabu_aspiration(P.st, 8 * n, n)
        x, g, E = P.state()
        T, Cm = I.icd2s_get_tabu(P.st, 1, n)
        xo, Eo, To, Co, _ = orc.tabu_asp(P.Q, X0[0], 8 * n, n)
        assert np.array_equal(x[0], xo) and E[0] == Eo, seed
        assert np.array_equal(T[0], To) and np.array_equal(Cm[0], Co), seed
        P.close()


@pytest.mark.parametrize("asp", [0, 1])
def test_tabu_with_a_move_log_beyond_shared_memory(L, orc, asp):
    """alpha = 120 000 at n = 300: the move log (2 bytes a move) no longer fits
    a CTA's shared memory and goes to global memory; the search still equals
    the oracle's, and a later shorter search (log back in shared memory) too."""
    n, R, c = 300, 2, 7
    P = Problem(n, 0.5, 77, R=R)
    X0 = random_solutions(n, R, 78)
    for alpha in (120_000, 900):
        P.load(X0)
        (I.icd2s_tabu_aspiration if asp else I.icd2s_tabu)(P.st, alpha, c)
        _check_tabu(orc, P.Q, X0, alpha, c, asp, P.state() + I.icd2s_get_tabu(P.st, R, n))
    P.close()


# ----------------------------------------------------------------------------- Tabu keys
def _compact_shift(n, bound):
    """Shift of the one-reduction Tabu keys: the index field holds n itself
    (2^b > n), and g + 2^(31 - sh) must stay inside [1, 2^(32 - sh) - 2]."""
    sh = int(n).bit_length() + 1
    return sh if bound + 1 < (1 << (31 - sh)) else 0


def _pk_shift(Q, bound):
    """The same for the keys on parity labels (one CTA per replica): the index
    field holds the rank of a variable within its class of Q_jj mod 2."""
    odd = int((np.diag(Q).astype(np.int64) & 1).sum())
    sh = max(odd, Q.shape[0] - odd).bit_length() + 1
    return sh if bound + 1 < (1 << (31 - sh)) else 0


def _attained_bound(Q):
    """max_j max(|Q_jj - 2 N_j|, |Q_jj + 2 P_j|), P_j / N_j the positive /
    negative off-diagonal sums of column j in magnitude, and an x attaining
    it: column j's couplings of the sign that widens it on, x_j = 0."""
    Qi = Q.astype(np.int64)
    d = np.diag(Qi).copy()
    off = Qi - np.diag(d)
    P, N = np.clip(off, 0, None).sum(axis=0), np.clip(-off, 0, None).sum(axis=0)
    hi, lo = np.abs(d + 2 * P), np.abs(d - 2 * N)
    j = int(np.maximum(hi, lo).argmax())
    x = ((off[:, j] > 0) if hi[j] >= lo[j] else (off[:, j] < 0)).astype(np.uint8)
    x[j] = 0
    return int(max(hi[j], lo[j])), x


def _tabu_both_keys(P, X0, alpha, c, asp, variant=-1, cluster=0):
    """Runs the search with the compact keys (where the instance allows them)
    and with the wide keys, each with the signed row pairs (where the
    instance has them) and with the plain rows, from the same start; returns
    the four results."""
    out = []
    for wide in (0, 1):
        for rows in (1, 2):
            P.load(X0)
            I.icd2s_set_tuning(P.st, tabu_variant=variant, tabu_wide_keys=wide, tabu_rows=rows,
                               tabu_cluster=cluster)
            (I.icd2s_tabu_aspiration if asp else I.icd2s_tabu)(P.st, alpha, c)
            out.append(P.state() + I.icd2s_get_tabu(P.st, P.R, P.n))
    return out


def _check_tabu(orc, Q, X0, alpha, c, asp, res):
    x, g, E, T, Cm = res
    for p in range(X0.shape[0]):
        xo, Eo, To, Co, _ = orc.tabu_asp(Q, X0[p], alpha, c, aspiration=asp)
        assert np.array_equal(x[p], xo) and E[p] == Eo, p
        assert np.array_equal(T[p], To) and np.array_equal(Cm[p], Co), p
        assert np.array_equal(g[p], orc.gains(Q, xo)), p


@pytest.mark.parametrize("n,density,seed", [(40, 1.0, 2), (2500, 0.1, 3), (5000, 0.5, 4), (700, 1.0, 5)])
def test_gain_bound(L, orc, n, density, seed):
    """icd2s_qubo_gain_bound is the largest gain magnitude over every x: the
    oracle's gains of an x built to attain it reach it exactly, no gain of
    sampled solutions exceeds it, and it lies within 2 max_j sum_i |Q_ij|."""
    Q = make_qubo(n, density, seed)
    q = I.icd2s_qubo_create(Q)
    bound = I.icd2s_qubo_gain_bound(q)
    I.icd2s_qubo_destroy(q)
    want, worst = _attained_bound(Q)
    assert bound == want
    assert int(np.abs(orc.gains(Q, worst).astype(np.int64)).max()) == bound
    assert bound <= 2 * int(np.abs(Q.astype(np.int64)).sum(axis=0).max())
    for x in list(random_solutions(n, 4, seed)):
        assert int(np.abs(orc.gains(Q, x).astype(np.int64)).max()) <= bound


@pytest.mark.parametrize("n,density,variant,asp", [(700, 0.5, -1, 0), (700, 0.5, 1, 1), (2500, 0.1, -1, 0),
                                                   (2500, 0.1, -1, 1), (300, 1.0, 4, 0), (300, 1.0, 5, 1),
                                                   (64, 1.0, -1, 1)])
def test_tabu_compact_and_wide_keys(L, orc, n, density, variant, asp):
    """Instances whose gains fit one 32-bit key: the compact and the wide
    keys give the oracle's search, with and without aspiration."""
    R, alpha, c = 3, 3 * n, max(2, n // 40)
    P = Problem(n, density, 7 * n + 1, R=R)
    assert _compact_shift(n, I.icd2s_qubo_gain_bound(P.q)) > 0
    X0 = random_solutions(n, R, n + 17)
    for res in _tabu_both_keys(P, X0, alpha, c, asp, variant):
        _check_tabu(orc, P.Q, X0, alpha, c, asp, res)
    P.close()


@pytest.mark.parametrize("n,asp", [(300, 0), (300, 1), (2500, 0)])
def test_tabu_with_entries_of_minus_128(L, orc, n, asp):
    """-128 has no int8 negation, so such an instance makes no signed rows
    even when asked for them: the search still equals the oracle, through the
    plain rows."""
    Q = make_qubo(n, 0.3, 50 + n).astype(np.int16)
    rng = np.random.Generator(np.random.PCG64(51))
    for i, j in rng.integers(0, n, size=(25, 2)):
        Q[i, j] = Q[j, i] = -128
    Q = Q.astype(np.int8)
    R, alpha, c = 3, 3 * n, max(2, n // 50)
    q = I.icd2s_qubo_create(Q)
    st = I.icd2s_state_create(q, R, 5)
    assert I.icd2s_qubo_gain_bound(q) == _attained_bound(Q)[0]
    X0 = random_solutions(n, R, 52)
    try:
        I.icd2s_set_tuning(st, tabu_rows=2)
        I.icd2s_state_load(st, X0)
        (I.icd2s_tabu_aspiration if asp else I.icd2s_tabu)(st, alpha, c)
        res = I.icd2s_get_state(st, R, n) + I.icd2s_get_tabu(st, R, n)
        _check_tabu(orc, Q, X0, alpha, c, asp, res)
    finally:
        I.icd2s_state_destroy(st)
        I.icd2s_qubo_destroy(q)


@pytest.mark.parametrize("n,density,variant,asp", [(5000, 0.5, -1, 0), (5000, 0.5, -1, 1), (5000, 0.5, 5, 0),
                                                   (5000, 0.5, 1, 1), (4800, 0.6, 5, 1), (4800, 0.6, 1, 0)])
def test_tabu_parity_label_keys(L, orc, n, density, variant, asp):
    """Instances whose gain bound is too wide for the compact keys on indices
    but fits them on parity labels (Q relabeled with the even-diagonal
    variables first): that search and the wide keys' give the oracle's, with
    and without aspiration."""
    R, alpha, c = 3, n, max(2, n // 50)
    P = Problem(n, density, 7 * n + 1, R=R)
    bound = I.icd2s_qubo_gain_bound(P.q)
    assert _compact_shift(n, bound) == 0 and _pk_shift(P.Q, bound) > 0
    X0 = random_solutions(n, R, n + 19)
    for res in _tabu_both_keys(P, X0, alpha, c, asp, variant, cluster=1):
        _check_tabu(orc, P.Q, X0, alpha, c, asp, res)
    P.close()


@pytest.mark.parametrize("mode", ["ck", "pk"])
@pytest.mark.parametrize("extra", [0, 1])
def test_tabu_keys_at_the_gain_bound(L, orc, mode, extra):
    """n = 8192: a heavy variable h whose gain bound is the largest a 32-bit
    key takes -- 65534 on indices (14-bit index field, shift 15), 2^(31 - s)
    - 2 on parity labels (shift s from the larger class) -- or, with Q_hh one
    larger, one more (the next wider keys).  Q_hh = 126 + extra and positive
    couplings (entries of 127, the rest of 1) summing to (target - 126) / 2;
    the start puts h at its extreme gains +-(Q_hh + 2 P_h), so the keys span
    their whole range."""
    n, R, alpha, c, h = 8192, 2, 1500, 54, 5000
    Q = make_qubo(n, 0.0005, 91).astype(np.int16)
    Q[h, :] = 0
    Q[:, h] = 0
    Q[h, h] = 126 + extra
    if mode == "ck":
        target = 65534
    else:
        odd = int((np.diag(Q) & 1).sum())
        target = (1 << (31 - (max(odd, n - odd).bit_length() + 1))) - 2
    half = (target - 126) // 2
    k127, k1 = half // 127, half % 127
    rng = np.random.Generator(np.random.PCG64(92))
    nb = np.sort(rng.choice(np.setdiff1d(np.arange(n), [h]), k127 + k1, replace=False))
    Q[h, nb[:k127]] = 127
    Q[h, nb[k127:]] = 1
    Q[nb, h] = Q[h, nb]
    Q = Q.astype(np.int8)
    q = I.icd2s_qubo_create(Q)
    bound = I.icd2s_qubo_gain_bound(q)
    assert bound == target + extra == _attained_bound(Q)[0]
    if mode == "ck":
        assert (_compact_shift(n, bound) == 15) == (extra == 0) and _pk_shift(Q, bound) > 0
    else:
        assert _compact_shift(n, bound) == 0 and (_pk_shift(Q, bound) > 0) == (extra == 0)
    st = I.icd2s_state_create(q, R, 3)

    class _P:
        pass
    P = _P()
    P.st, P.R, P.n, P.q = st, R, n, q
    P.load = lambda X: I.icd2s_state_load(st, X)
    P.state = lambda: I.icd2s_get_state(st, R, n)
    X0 = random_solutions(n, R, 93)
    X0[:, nb] = 1
    X0[0, h], X0[1, h] = 0, 1          # the heavy variable's largest gain, and its negative
    assert int(orc.gains(Q, X0[0])[h]) == bound and int(orc.gains(Q, X0[1])[h]) == -bound
    try:
        for asp in (0, 1):
            for cluster in (1, 0):     # one CTA per replica, and the default split (n >= 8192, R = 2)
                for res in _tabu_both_keys(P, X0, alpha, c, asp, cluster=cluster):
                    _check_tabu(orc, Q, X0, alpha, c, asp, res)
    finally:
        I.icd2s_state_destroy(st)
        I.icd2s_qubo_destroy(q)


# ----------------------------------------------------------------------------- Algorithm 1 on a cluster
@pytest.mark.parametrize("G", [1, 2, 4])
@pytest.mark.parametrize("n,density,asp,wide,alpha,c,R", [
    (300, 0.5, 0, 0, 900, 3, 3),      # slices of 128 / 256 variables, the last one ragged
    (300, 0.5, 1, 1, 900, 60, 2),     # aspiration, wide keys
    (2500, 0.1, 0, 0, 2000, 16, 3),   # compact keys
    (2500, 0.1, 1, 0, 3000, 40, 2),
    (5000, 0.5, 0, 1, 2000, 33, 2),   # the time-to-target instance: wide keys
    (5000, 0.5, 1, 1, 2000, 120, 2),
    (700, 1.0, 1, 0, 2100, 17, 3),
    (40, 1.0, 1, 0, 320, 40, 2),      # c = n: the all-tabu fallback; CTAs with no variables
    (13001, 0.5, 0, 1, 150, 86, 1),
])
def test_tabu_split_over_a_cluster(L, orc, G, n, density, asp, wide, alpha, c, R):
    """Algorithm 1 with every replica's variables split over a cluster of G
    CTAs (the per-move arg-min exchanged through distributed shared memory):
    the search equals the oracle's for every G, with and without aspiration
    and with compact and wide keys."""
    P = Problem(n, density, 3 * n + 1, R=R)
    X0 = random_solutions(n, R, n + c)
    P.load(X0)
    I.icd2s_set_tuning(P.st, tabu_cluster=G, tabu_wide_keys=wide)
    (I.icd2s_tabu_aspiration if asp else I.icd2s_tabu)(P.st, alpha, c)
    _check_tabu(orc, P.Q, X0, alpha, c, asp, P.state() + I.icd2s_get_tabu(P.st, R, n))
    P.close()


@pytest.mark.parametrize("G,asp", [(2, 0), (4, 1)])
def test_tabu_split_with_a_move_log_beyond_shared_memory(L, orc, G, asp):
    """The cluster split with the move log in global memory (written by the
    cluster's first CTA, read by all after the search)."""
    n, R, c = 300, 2, 7
    P = Problem(n, 0.5, 79, R=R)
    X0 = random_solutions(n, R, 80)
    I.icd2s_set_tuning(P.st, tabu_cluster=G)
    for alpha in (120_000, 900):
        P.load(X0)
        (I.icd2s_tabu_aspiration if asp else I.icd2s_tabu)(P.st, alpha, c)
        _check_tabu(orc, P.Q, X0, alpha, c, asp, P.state() + I.icd2s_get_tabu(P.st, R, n))
    P.close()


@pytest.mark.parametrize("G,variant", [(2, 4), (4, 5), (2, 1)])
def test_tabu_split_in_other_kernel_shapes(L, orc, G, variant):
    n, R, alpha, c = 2500, 2, 1500, 16
    P = Problem(n, 0.1, 81, R=R)
    X0 = random_solutions(n, R, 82)
    P.load(X0)
    I.icd2s_set_tuning(P.st, tabu_cluster=G, tabu_variant=variant)
    I.icd2s_tabu(P.st, alpha, c)
    _check_tabu(orc, P.Q, X0, alpha, c, 0, P.state() + I.icd2s_get_tabu(P.st, R, n))
    P.close()


def test_tabu_cluster_setting_is_checked(L):
    P = Problem(300, 0.5, 1, R=2)
    with pytest.raises(I.ICD2SError):
        I.icd2s_set_tuning(P.st, tabu_cluster=3)
    with pytest.raises(I.ICD2SError):
        I.icd2s_set_tuning(P.st, tabu_cluster=2, tabu_variant=3)   # a one-CTA-only shape
    P.close()


# ----------------------------------------------------------------------------- Eq. 6-8, Alg. 3, selection
@pytest.mark.parametrize("n,R,K,m_min,m_max", [(500, 6, 3, 8, 40), (333, 4, 1, 64, 64), (2500, 3, 16, 32, 150)])
def test_control_parameters_and_selection(L, orc, n, R, K, m_min, m_max):
    torch = torch_cuda()
    P = Problem(n, 0.5, 7, R=R, state_seed=99)
    X0 = random_solutions(n, R, 1)
    P.load(X0)
    I.icd2s_tabu(P.st, 3 * n, 3)
    x, _, _ = P.state()
    T, _ = I.icd2s_get_tabu(P.st, R, n)
    it = 5
    sp = I.SelectParams(w1=65536, w2=65536, w3=32768, K=K, m_min=m_min, m_max=m_max, iter=it)
    idx = torch.zeros(R * K * m_max + 1, dtype=torch.int32, device="cuda")
    off = torch.zeros(R * K + 1, dtype=torch.int32, device="cuda")
    I.icd2s_select_subqubos(P.st, sp, idx.data_ptr(), off.data_ptr())
    A, gam, dl = I.icd2s_get_control(P.st, R, n)
    idx, off = idx.cpu().numpy(), off.cpu().numpy()
    gam_o = orc.gamma(x)
    assert np.array_equal(gam, gam_o)
    eh = orc.eta_hat(orc.eta(P.Q))
    for p in range(R):
        d_o = orc.delta(T[p])
        A_o = orc.aggregate(eh, gam_o, d_o)
        assert np.array_equal(dl[p], d_o) and np.array_equal(A[p], A_o)
        sizes = orc.subqubo_sizes(K, m_min, m_max, 99, p, it)
        assert np.array_equal(np.diff(off[p * K:(p + 1) * K + 1]), sizes)
        got = idx[off[p * K]:off[(p + 1) * K]]
        assert np.array_equal(got, orc.select(A_o, sizes))
    P.close()


# ----------------------------------------------------------------------------- Eq. 4, Algorithm 4
SIZES = [1, 5, 16, 31, 32, 33, 64, 65, 100, 128, 129, 200, 256]


@pytest.mark.parametrize("scheme", [1, 2, 3, 4])
@pytest.mark.parametrize("sweeps,T_max,density", [(1, 50.0, 1.0), (7, 400.0, 1.0), (64, 2000.0, 1.0),
                                                   (64, 3000.0, 0.05), (32, 800.0, 0.2)])
def test_anneal(L, orc, sweeps, T_max, density, scheme):
    """Every sweep scheme (rounds of decisions, position by position,
    position by position with both outcomes of the next test, and the choice
    per sweep) gives the sequential Metropolis sweep.  Dense subQUBOs take one accept per round;
    sparse ones (5 %, 20 %) exercise the rounds of several uncoupled
    accepts."""
    torch = torch_cuda()
    n, R, it = 2000, 3, 17
    K = len(SIZES) // R + 1
    P = Problem(n, density, 21, R=R, state_seed=1234)
    I.icd2s_set_tuning(P.st, anneal_scheme=scheme)
    X0 = random_solutions(n, R, 2)
    P.load(X0)
    groups, offs = [], [0]
    count = 0
    for p in range(R):
        sz = [SIZES[(p * K + k) % len(SIZES)] for k in range(K)]
        g = random_subsets(n, sz, 100 + p)
        off = 0
        for m in sz:
            groups.append((p, g[off:off + m]))
            offs.append(offs[-1] + m)
            off += m
            count += 1
    idx = np.concatenate([g for _, g in groups]).astype(np.int32)
    off = np.array(offs, np.int32)
    mask = torch.zeros((R, n), dtype=torch.uint8, device="cuda")
    dE = torch.zeros(count, dtype=torch.int64, device="cuda")
    ap = I.AnnealParams(sweeps=sweeps, T_max=T_max, T_min=1.0, iter=it, per_replica=K)
    idx_d, off_d = dev(idx), dev(off)   # keep the tensors alive while the library uses them
    I.icd2s_anneal_subqubos_batch(P.st, idx_d.data_ptr(), off_d.data_ptr(), count, ap, mask.data_ptr(),
                                  dE.data_ptr())
    mask, dE = mask.cpu().numpy(), dE.cpu().numpy()
    beta = orc.beta_table(sweeps, T_max, 1.0)
    nlog = orc.nlog_table()
    want = np.zeros((R, n), np.uint8)
    for s, (p, S) in enumerate(groups):
        Qs, _ = orc.subqubo(P.Q, X0[p], S)
        xs1, dEo, _ = orc.anneal(Qs, X0[p][S], beta, nlog, 1234, s, it)
        want[p, S] = xs1 != X0[p][S]
        assert dE[s] == dEo, (s, len(S))
    assert np.array_equal(mask, want)
    x, _, _ = P.state()
    assert np.array_equal(x, X0)  # the anneal call leaves the solutions alone
    P.close()


@pytest.mark.parametrize("density", [1.0, 0.1])
def test_exact_subqubos(L, orc, density):
    """Exact Ising machine (all 2^m assignments, Gray-code walk split over the
    lanes) against the oracle's brute force, m = 1..20 (fewer than 32 lanes
    for m < 5, one dynamic flip per 16 steps for m >= 9)."""
    torch = torch_cuda()
    n, R, K = 600, 3, 3
    sizes = [1, 3, 4, 5, 6, 8, 13, 16, 20]
    P = Problem(n, density, 33, R=R, state_seed=77)
    X0 = random_solutions(n, R, 5)
    P.load(X0)
    groups, offs = [], [0]
    for p in range(R):
        sz = sizes[p * K:(p + 1) * K]
        g = random_subsets(n, sz, 200 + p)
        o = 0
        for m in sz:
            groups.append((p, g[o:o + m]))
            offs.append(offs[-1] + m)
            o += m
    idx_d = dev(np.concatenate([g for _, g in groups]).astype(np.int32))
    off_d = dev(np.array(offs, np.int32))
    mask = torch.zeros((R, n), dtype=torch.uint8, device="cuda")
    dE = torch.zeros(len(groups), dtype=torch.int64, device="cuda")
    I.icd2s_exact_subqubos_batch(P.st, idx_d.data_ptr(), off_d.data_ptr(), len(groups), K, mask.data_ptr(),
                                 dE.data_ptr())
    mask, dE = mask.cpu().numpy(), dE.cpu().numpy()
    want = np.zeros((R, n), np.uint8)
    for s_, (p, S) in enumerate(groups):
        Qs, _ = orc.subqubo(P.Q, X0[p], S)
        y, dEo = orc.exact_subqubo(Qs, X0[p][S])
        want[p, S] = y != X0[p][S]
        assert dE[s_] == dEo, (s_, len(S))
    assert np.array_equal(mask, want)
    P.close()


def test_exact_subqubo_m24_is_a_local_optimum_below_annealing(L, orc):
    """m = 22 and 24 (too large for the oracle's brute force): no single flip
    of the returned assignment lowers the subQUBO objective, and it is not
    above a slow anneal of the same subQUBO."""
    torch = torch_cuda()
    n = 300
    P = Problem(n, 1.0, 44, R=1, state_seed=3)
    X0 = random_solutions(n, 1, 8)
    P.load(X0)
    for m in (22, 24):
        S = np.sort(random_subsets(n, [m], 9 + m)).astype(np.int32)
        idx_d, off_d = dev(S), dev(np.array([0, m], np.int32))
        mask = torch.zeros((1, n), dtype=torch.uint8, device="cuda")
        dE = torch.zeros(1, dtype=torch.int64, device="cuda")
        I.icd2s_exact_subqubos_batch(P.st, idx_d.data_ptr(), off_d.data_ptr(), 1, 1, mask.data_ptr(), dE.data_ptr())
        Qs, _ = orc.subqubo(P.Q, X0[0], S)
        y = X0[0][S] ^ mask.cpu().numpy()[0][S]
        f = orc.subqubo_energy(Qs, y)
        assert f - orc.subqubo_energy(Qs, X0[0][S]) == int(dE.cpu()[0])
        for a in range(m):
            y2 = y.copy()
            y2[a] ^= 1
            assert orc.subqubo_energy(Qs, y2) >= f
        x1, dEa, _ = orc.anneal(Qs, X0[0][S], orc.beta_table(300, 3000.0, 0.5), orc.nlog_table(), 1, 0, 0)
        assert f <= orc.subqubo_energy(Qs, x1)
    P.close()


def test_anneal_rejects_oversized_subqubos(L):
    torch = torch_cuda()
    P = Problem(600, 1.0, 1, R=1)
    off = dev(np.array([0, 257], np.int32))
    idx = dev(np.arange(257, dtype=np.int32))
    mask = torch.zeros((1, 600), dtype=torch.uint8, device="cuda")
    with pytest.raises(I.ICD2SError) as e:
        I.icd2s_anneal_subqubos_batch(P.st, idx.data_ptr(), off.data_ptr(), 1,
                                      I.AnnealParams(sweeps=4, T_max=10.0, T_min=1.0, iter=0, per_replica=1),
                                      mask.data_ptr())
    assert e.value.code == I.ERR_RANGE
    P.close()


# ----------------------------------------------------------------------------- write-back
@pytest.mark.parametrize("n,R", [(64, 2), (1000, 5), (2500, 4), (3000, 3)])
def test_apply_flips_update_gains(L, orc, n, R):
    P = Problem(n, 0.7, n, R=R)
    X0 = random_solutions(n, R, 9)
    P.load(X0)
    rng = np.random.default_rng(n)
    M = np.zeros((R, n), np.uint8)
    M[0] = 0                                            # nothing flips
    M[1] = rng.random(n) < 0.02
    if R > 2:
        M[2] = 1                                        # everything flips
    for p in range(3, R):
        M[p] = rng.random(n) < 0.3
    M_d = dev(M)
    I.icd2s_apply_flips_update_gains(P.st, M_d.data_ptr())
    x, g, E = P.state()
    X1 = X0 ^ M
    assert np.array_equal(x, X1)
    assert np.array_equal(E, orc.energy_batch(P.Q, X1))
    for p in range(R):
        assert np.array_equal(g[p], orc.gains(P.Q, X1[p]))
    # a second round on the updated state
    M2_d = dev(M[::-1].copy())
    I.icd2s_apply_flips_update_gains(P.st, M2_d.data_ptr())
    x, g, E = P.state()
    X2 = X1 ^ M[::-1]
    assert np.array_equal(x, X2) and np.array_equal(E, orc.energy_batch(P.Q, X2))
    P.close()


# ----------------------------------------------------------------------------- mutation
@pytest.mark.parametrize("mode,rate,t", [(0, 0.0, 3), (1, 0.3, 8), (0, 0.0, 15), (1, 1.0, 1)])
def test_mutate(L, orc, mode, rate, t):
    torch = torch_cuda()
    n, R, K, m_min, m_max = 700, 4, 2, 20, 60
    P = Problem(n, 0.4, 3, R=R, state_seed=77)
    X0 = random_solutions(n, R, 4)
    P.load(X0)
    I.icd2s_tabu(P.st, 2 * n, 4)
    x1, _, _ = P.state()
    T, _ = I.icd2s_get_tabu(P.st, R, n)
    sp = I.SelectParams(w1=65536, w2=65536, w3=32768, K=K, m_min=m_min, m_max=m_max, iter=t)
    idx = torch.zeros(R * K * m_max + 1, dtype=torch.int32, device="cuda")
    off = torch.zeros(R * K + 1, dtype=torch.int32, device="cuda")
    I.icd2s_select_subqubos(P.st, sp, idx.data_ptr(), off.data_ptr())
    mask = torch.zeros((R, n), dtype=torch.uint8, device="cuda")
    I.icd2s_mutate(P.st, I.MutateParams(mut_mode=mode, mut_rate=rate, iter=t), mask.data_ptr())
    x2, g2, E2 = P.state()
    mask = mask.cpu().numpy()
    eh = orc.eta_hat(orc.eta(P.Q))
    gam = orc.gamma(x1)
    r = orc.mutation_rate(t) if mode == 0 else rate
    for p in range(R):
        A = orc.aggregate(eh, gam, orc.delta(T[p]))
        sizes = orc.subqubo_sizes(K, m_min, m_max, 77, p, t)
        sel = np.zeros(n, np.uint8)
        sel[orc.select(A, sizes)] = 1
        L_ = int(np.floor((n - sizes.sum()) * r))
        xo, _ = orc.mutate(A, sel, L_, 77, p, t, x1[p])
        assert np.array_equal(x2[p], xo), p
        assert np.array_equal(mask[p], (xo != x1[p]).astype(np.uint8))
        assert E2[p] == orc.energy(P.Q, xo)
        assert np.array_equal(g2[p], orc.gains(P.Q, xo))
    P.close()


def test_mutate_before_select_is_an_error(L):
    P = Problem(100, 1.0, 1, R=2)
    with pytest.raises(I.ICD2SError) as e:
        I.icd2s_mutate(P.st, I.MutateParams(mut_mode=0, mut_rate=0.0, iter=0))
    assert e.value.code == I.ERR_STATE
    P.close()


# ----------------------------------------------------------------------------- Call_IM_Solution_Set
@pytest.mark.parametrize("n,z,m,K,order,im_mode", [(64, 8, 16, 1, 0, 0), (300, 3, 40, 1, 0, 0), (1000, 2, 64, 1, 0, 0),
                                                   (1000, 3, 64, 4, 0, 0), (1000, 3, 64, 4, 1, 0),
                                                   (2500, 5, 64, 16, 0, 0), (300, 3, 20, 3, 0, 1)])
def test_initial_pass(L, orc, n, z, m, K, order, im_mode):
    """One block at a time, and K blocks at once with K Ising machines per
    solution (the last group shorter: 15 blocks in groups of 4, 39 in groups
    of 16), annealed or solved exactly."""
    P = Problem(n, 1.0, 8, R=z, state_seed=5)
    lp = lib_params(I, n, z=z, K=K, m_min=m, m_max=m, m_init=m, sweeps=32, T_max=500.0, im_order=order,
                    im_mode=im_mode)
    I.icd2s_initial_pass(P.st, lp)
    x, g, E = P.state()
    S0 = orc.init_solutions(n, z, 5)
    So, Eo = orc.initial_pass(P.Q, orc_params(orc, lp), 5, S0)
    assert np.array_equal(x, So) and np.array_equal(E, Eo)
    P.close()


# ----------------------------------------------------------------------------- kernel variants
@pytest.mark.parametrize("variant", range(6))
def test_every_tabu_variant_gives_the_same_search(L, orc, variant):
    n, R, alpha, c = 700, 3, 900, 5
    P = Problem(n, 0.5, 12, R=R)
    try:
        I.icd2s_set_tuning(P.st, tabu_variant=variant)
    except I.ICD2SError as e:
        assert e.code == I.ERR_ARG  # the variant cannot cover n with its block size
        P.close()
        return
    X0 = random_solutions(n, R, 13)
    P.load(X0)
    I.icd2s_tabu(P.st, alpha, c)
    x, g, E = P.state()
    T, Cm = I.icd2s_get_tabu(P.st, R, n)
    for p in range(R):
        xo, Eo, To, Co = orc.tabu(P.Q, X0[p], alpha, c)
        assert np.array_equal(x[p], xo) and E[p] == Eo
        assert np.array_equal(T[p], To) and np.array_equal(Cm[p], Co)
        assert np.array_equal(g[p], orc.gains(P.Q, xo))
    P.close()


def test_autotune_keeps_the_state_and_the_results(L, orc):
    n, z = 900, 6
    P = Problem(n, 0.3, 4, R=z, state_seed=21)
    lp = lib_params(I, n, z=z, K=2, m_min=20, m_max=100, m_init=50, alpha=2 * n, c=6, sweeps=40, T_max=900.0)
    S0 = random_solutions(n, z, 8)
    P.load(S0)
    x0, g0, E0 = P.state()
    choice = I.icd2s_autotune(P.st, lp)
    assert choice == I.icd2s_get_tuning(P.st)
    x1, g1, E1 = P.state()
    assert np.array_equal(x0, x1) and np.array_equal(g0, g1) and np.array_equal(E0, E1)
    I.icd2s_step(P.st, lp, 0)
    x, g, E = P.state()
    o = orc.step(P.Q, orc_params(orc, lp), 21, 0, S0)
    assert np.array_equal(x, o["S"]) and np.array_equal(E, o["E"])
    P.close()
