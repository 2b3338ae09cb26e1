"""Pins of the oracle's learned-selection parts (the proposal network added to
IC-D2S, readings S21/S22): the features against a hand-worked example, the
double network against torch autograd and finite differences, closed forms
of the loss, the float score against the double one within its rounding
bound, the BF16 rounding against torch, and the learned step against
selections with a known answer.  No GPU."""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import mlp_ref as M
from paper_2502_13947_gb300.instances import make_qubo, random_solutions

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _rand_weights(seed, scale=0.3):
    rng = np.random.default_rng(seed)
    W = rng.uniform(-scale, scale, M.NPAR).astype(np.float32)
    return M.bf16_round(W)


def _rand_features(seed, rows):
    rng = np.random.default_rng(seed)
    F = np.empty((rows, 6), np.float32)
    F[:, 0] = rng.integers(0, 2, rows)
    F[:, 1] = rng.uniform(-1, 1, rows)
    F[:, 2:] = rng.uniform(0, 1, (rows, 4))
    return F


# ----------------------------------------------------------------------------- features
def test_features_hand_worked(orc):
    with open(os.path.join(GOLD, "features3_worked.json")) as f:
        g = json.load(f)
    F = orc.features(np.array(g["x"]), np.array(g["g"]), np.array(g["T"]), np.array(g["C"]),
                     np.array(g["H"]), np.array(g["eta_hat"]), g["t"], g["alpha"], g["c"])
    exp = np.array([[np.float32(float(Fraction(a, b))) for a, b in row] for row in g["expected"]], np.float32)
    assert F.dtype == np.float32 and F.shape == (3, 6)
    assert np.array_equal(F, exp)


def test_features_zero_alpha_and_ranges(orc):
    rng = np.random.default_rng(3)
    n = 50
    x = rng.integers(0, 2, n)
    g = rng.integers(-5000, 5000, n)
    T = np.zeros(n, np.int32)
    Cm = rng.integers(0, 7, n)
    H = rng.integers(0, 10, n)
    eh = rng.integers(0, 65537, n)
    F = orc.features(x, g, T, Cm, H, eh, 9, 0, 7)
    assert np.all(F[:, 2] == 0)                     # alpha = 0
    assert np.all(np.abs(F[:, 1]) < 1)              # |g| / (max|g| + 1) < 1
    assert np.all((F[:, 3] >= 0) & (F[:, 3] <= 1))
    assert np.all((F[:, 4] >= 0) & (F[:, 4] <= 1))
    assert np.all((F[:, 5] >= 0) & (F[:, 5] <= 1))


# ----------------------------------------------------------------------------- BF16 rounding
def test_bf16_round_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    a = np.concatenate([rng.normal(0, 1, 5000), rng.normal(0, 1e-3, 1000), rng.normal(0, 1e4, 1000)]).astype(np.float32)
    # exact ties: 1 + 2^-8 rounds down to 1 (even), 1 + 3 * 2^-8 up to 1 + 2^-6
    a = np.concatenate([a, np.array([1 + 2 ** -8, 1 + 3 * 2 ** -8, -(1 + 2 ** -8), 0.0, -0.0], np.float32)])
    ref = torch.from_numpy(a).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(M.bf16_round(a).view(np.uint32), ref.view(np.uint32))
    assert M.bf16_round(np.float32(1 + 2 ** -8)) == 1.0
    assert M.bf16_round(np.float32(1 + 3 * 2 ** -8)) == np.float32(1 + 2 ** -6)


# ----------------------------------------------------------------------------- double network
def test_network_matches_torch_autograd():
    torch = pytest.importorskip("torch")
    W = _rand_weights(1).astype(np.float64)
    F = _rand_features(2, 97)
    y = (np.random.default_rng(3).uniform(size=97) < 0.2).astype(np.float64)
    L, grad = M.loss_and_grad(W, F, y, pos_weight=3.0)
    Wt = torch.tensor(W, dtype=torch.float64, requires_grad=True)
    W1 = Wt[M.OFF_W1:M.OFF_B1].view(64, 6)
    b1 = Wt[M.OFF_B1:M.OFF_W2]
    W2 = Wt[M.OFF_W2:M.OFF_B2].view(64, 64)
    b2 = Wt[M.OFF_B2:M.OFF_W3]
    w3 = Wt[M.OFF_W3:M.OFF_B3]
    b3 = Wt[M.OFF_B3]
    Ft = torch.tensor(F, dtype=torch.float64)
    h = torch.relu(torch.relu(Ft @ W1.T + b1) @ W2.T + b2)
    s = h @ w3 + b3
    lt = torch.nn.functional.binary_cross_entropy_with_logits(
        s, torch.tensor(y), pos_weight=torch.tensor(3.0, dtype=torch.float64))
    lt.backward()
    assert abs(float(lt.detach()) - L) < 1e-12
    np.testing.assert_allclose(grad, Wt.grad.numpy(), rtol=1e-10, atol=1e-13)
    np.testing.assert_allclose(M.forward(W, F)[0], s.detach().numpy(), rtol=1e-12, atol=1e-12)


def test_gradient_finite_differences():
    W = _rand_weights(4).astype(np.float64)
    F = _rand_features(5, 40)
    y = (np.random.default_rng(6).uniform(size=40) < 0.3).astype(np.float64)
    _, grad = M.loss_and_grad(W, F, y, pos_weight=2.0)
    rng = np.random.default_rng(7)
    idx = np.concatenate([rng.choice(M.NPAR, 200, replace=False), [M.OFF_B3, M.OFF_W1, M.OFF_B1, M.OFF_W3]])
    h = 1e-6
    for i in idx:
        Wp, Wm = W.copy(), W.copy()
        Wp[i] += h
        Wm[i] -= h
        fd = (M.loss(Wp, F, y, 2.0) - M.loss(Wm, F, y, 2.0)) / (2 * h)
        assert abs(fd - grad[i]) <= 1e-7 + 1e-5 * abs(grad[i]), i


def test_zero_network_closed_form():
    W = np.zeros(M.NPAR)
    W[M.OFF_B3] = 0.75
    F = _rand_features(8, 33)
    y = np.zeros(33)
    y[:11] = 1
    pw = 2.5
    L, grad = M.loss_and_grad(W, F, y, pw)
    sp = lambda v: np.log1p(np.exp(v))
    sig = 1 / (1 + np.exp(-0.75))
    assert abs(L - (pw * (11 / 33) * sp(-0.75) + (22 / 33) * sp(0.75))) < 1e-14
    assert abs(grad[M.OFF_B3] - (pw * (11 / 33) * (sig - 1) + (22 / 33) * sig)) < 1e-14
    grad[M.OFF_B3] = 0
    assert np.all(grad == 0)


def test_adam_first_step_is_signed_lr():
    rng = np.random.default_rng(9)
    w = rng.normal(size=100)
    g = rng.normal(size=100)
    w1, m, v = M.adam(w, np.zeros(100), np.zeros(100), g, 1, lr=1e-3)
    np.testing.assert_allclose(w1, w - 1e-3 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    np.testing.assert_allclose(m, 0.1 * g)
    np.testing.assert_allclose(v, 0.001 * g * g)


# ----------------------------------------------------------------------------- float score
def test_float_score_single_path_exact(orc):
    W = np.zeros(M.NPAR, np.float32)
    W[M.OFF_W1 + 0 * 6 + 1] = -2.0          # a1_0 = -2 f1 + 0.5
    W[M.OFF_B1 + 0] = 0.5
    W[M.OFF_W2 + 3 * 64 + 0] = 1.5          # a2_3 = 1.5 h1_0 - 0.25
    W[M.OFF_B2 + 3] = -0.25
    W[M.OFF_W3 + 3] = 4.0
    W[M.OFF_B3] = -1.0
    F = np.array([[0, -0.25, 0, 0, 0, 0], [0, 0.5, 0, 0, 0, 0], [1, 0.125, 1, 1, 1, 1]], np.float32)
    # f1 = -0.25: h1 = 1, h2 = 1.25, s = 4; f1 = 0.5: h1 = 0, h2 = 0, s = -1;
    # f1 = 0.125: h1 = 0.25, a2 = 0.125, s = -0.5
    assert orc.mlp_score_f32(W, F).tolist() == [4.0, -1.0, -0.5]


def test_float_score_within_bound_of_double(orc):
    W = _rand_weights(10)
    F = _rand_features(11, 300)
    s32 = orc.mlp_score_f32(W, F)
    s64, (_, _, h1, _, h2) = M.forward(W, F)
    # each of the 2 x 64-term float sums adds at most ~64 ulps of its magnitude
    bound = 1e-4 * (1 + np.abs(s64))
    assert np.all(np.abs(s32 - s64) <= bound)


def test_score_key_is_monotone(orc):
    vals = np.array([-np.inf, -3e38, -2.0, -1.0, -1e-30, -1e-45, -0.0, 0.0, 1e-45, 1e-30, 0.5, 1.0, 2.0,
                     3e38, np.inf], np.float32)
    keys = [orc.score_key(v) for v in vals]
    assert all(a < b for a, b in zip(keys, keys[1:]))
    assert orc.score_key(0.0) == 0 and orc.score_key(-0.0) == -1


# ----------------------------------------------------------------------------- learned step
def _setup(n=48, z=4, K=2, m_min=5, m_max=9, seed=21):
    from oracle import oracle as o
    Q = make_qubo(n, 0.6, seed)
    prm = o.default_params(n, z=z, K=K, m_min=m_min, m_max=m_max, m_init=8, alpha=2 * n, c=3, sweeps=16,
                           T_max=60.0, max_iters=3)
    S = random_solutions(n, z, seed + 1)
    return o, Q, prm, S


def test_constant_network_selects_lowest_indices():
    o, Q, prm, S = _setup()
    prm.select_mode = 1
    W = np.zeros(M.NPAR, np.float32)
    r = o.step(Q, prm, 77, 2, S, H=np.zeros(S.shape, np.int32), W=W)
    for p in range(prm.z):
        sizes = o.subqubo_sizes(prm.K, prm.m_min, prm.m_max, 77, p, 2)
        Mp = int(np.sum(sizes))
        assert r["H"][p, :Mp].tolist() == [1] * Mp and not r["H"][p, Mp:].any()


def test_eta_network_selects_like_eta_ranking():
    o, Q, prm, S = _setup(seed=31)
    prm.select_mode = 1
    W = np.zeros(M.NPAR, np.float32)
    W[M.OFF_W1 + 0 * 6 + 5] = 1.0           # s = relu(relu(f5)) = eta_hat / 2^16, exactly
    W[M.OFF_W2 + 0] = 1.0
    W[M.OFF_W3 + 0] = 1.0
    eh = o.eta_hat(o.eta(Q))
    r = o.step(Q, prm, 5, 0, S, H=np.zeros(S.shape, np.int32), W=W, want_features=True)
    assert np.array_equal(r["score"], np.broadcast_to((eh / 65536.0).astype(np.float32), r["score"].shape))
    for p in range(prm.z):
        sizes = o.subqubo_sizes(prm.K, prm.m_min, prm.m_max, 5, p, 0)
        sel = np.sort(o.select(eh, sizes))
        assert np.flatnonzero(r["H"][p]).tolist() == sel.tolist()


def test_hybrid_mode_keeps_plain_rows():
    o, Q, prm, S = _setup(z=6, seed=41)
    W = _rand_weights(12)
    H0 = np.random.default_rng(1).integers(0, 3, S.shape).astype(np.int32)
    plain = o.step(Q, prm, 9, 4, S, H=H0, W=W)
    prm.select_mode = 2
    hyb = o.step(Q, prm, 9, 4, S, H=H0, W=W)
    # odd solutions keep the A ranking; every phase of one solution depends on
    # the others only through gamma, which is taken before the selection
    assert np.array_equal(hyb["S"][1::2], plain["S"][1::2])
    assert np.array_equal(hyb["H"][1::2], plain["H"][1::2])
    assert np.array_equal(hyb["T"], plain["T"]) and np.array_equal(hyb["A"], plain["A"])


def test_plain_step_ignores_network_and_reports_features():
    o, Q, prm, S = _setup(seed=51)
    a = o.step(Q, prm, 3, 1, S)
    b = o.step(Q, prm, 3, 1, S, W=_rand_weights(13), want_features=True)
    assert np.array_equal(a["S"], b["S"]) and a["best_E"] == b["best_E"]
    eh = o.eta_hat(o.eta(Q))
    # features of solution 0 at selection time: recompute from the post-Tabu state
    x0 = S[0].copy()
    xt, _, T, Cm = o.tabu(Q, x0, prm.alpha, prm.c)
    F0 = o.features(xt, o.gains(Q, xt), T, Cm, np.zeros(Q.shape[0], np.int32), eh, 1, prm.alpha, prm.c)
    assert np.array_equal(b["F"][0], F0)
    assert np.array_equal(b["score"][0], o.mlp_score_f32(_rand_weights(13), F0))
