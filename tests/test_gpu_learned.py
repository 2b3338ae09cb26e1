"""GPU parity of the learned selection (the proposal network added to the
method's choice of S'): features, scores, hit counts, the improvement log and
whole learned trajectories equal the oracle's bit for bit; the network's
scores and gradients agree with the double-precision reference within 1e-3;
the Adam step equals its definition; training on the GPU lowers the loss."""
import numpy as np
import pytest

from oracle import mlp_ref as M
from paper_2502_13947_gb300 import build as B
from paper_2502_13947_gb300 import icd2s as I
from paper_2502_13947_gb300.instances import make_qubo

from .gpu_util import dev, lib_params, orc_params, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    torch_cuda()
    B.build()
    return I.lib()


def _weights(seed, scale=0.3):
    return np.random.default_rng(seed).uniform(-scale, scale, M.NPAR).astype(np.float32)


def _features(seed, rows):
    rng = np.random.default_rng(seed)
    F = np.empty((rows, 6), np.float32)
    F[:, 0] = rng.integers(0, 2, rows)
    F[:, 1] = rng.uniform(-1, 1, rows)
    F[:, 2:] = rng.uniform(0, 1, (rows, 4))
    return F


def _oracle_chain(orc, Q, op, seed, iters, W=None):
    """Algorithm 2 in the oracle, one step at a time, with hit counts, the
    features at selection time and the improvement log (entries: features of
    the winning solution, best_x XOR the best at the previous entry)."""
    n = Q.shape[0]
    S = orc.init_solutions(n, op.z, seed)
    S, E = orc.initial_pass(Q, op, seed, S)
    b = int(np.argmin(E))
    best_E, best_x = int(E[b]), S[b].copy()
    H = np.zeros((op.z, n), np.int32)
    prev = best_x.copy()
    steps, log = [], []
    for t in range(iters):
        r = orc.step(Q, op, seed, t, S, best_E, best_x, H=H, W=W, want_features=True)
        if r["improved"]:
            log.append((r["F"][r["winner"]].copy(), r["best_x"] ^ prev, r["winner"]))
            prev = r["best_x"].copy()
        S, best_E, best_x, H = r["S"], r["best_E"], r["best_x"], r["H"]
        steps.append(r)
    return steps, log


def _net(Wf):
    m = I.icd2s_mlp_create(11)
    I.icd2s_mlp_set_weights(m, Wf)
    return m, I.icd2s_mlp_get_weights(m)[1]


@pytest.mark.parametrize("mode,order", [(1, 0), (2, 0), (1, 1)])
def test_learned_steps_equal_oracle(L, orc, mode, order):
    """n = 200 (ragged against the 128-wide rows), 6 replicas x 2 uneven
    subQUBOs (merged, or in Gauss-Seidel order): per step the features,
    scores, hit counts, solutions and energies equal the oracle's."""
    n, seed = 200, 5
    Q = make_qubo(n, 0.4, 77)
    lp = lib_params(I, n, z=6, K=2, m_min=8, m_max=20, m_init=20, alpha=2 * n, c=3, sweeps=32, T_max=400.0,
                    mut_mode=0, patience=0, max_iters=4, select_mode=mode, im_order=order)
    op = orc_params(orc, lp)
    m, Wb = _net(_weights(3))
    steps, _ = _oracle_chain(orc, Q, op, seed, 4, W=Wb)
    q = I.icd2s_qubo_create(Q)
    st = I.icd2s_state_create(q, lp.z, seed)
    try:
        I.icd2s_state_set_mlp(st, m)
        I.icd2s_initial_pass(st, lp)
        I.icd2s_best_update(st)
        for t, r in enumerate(steps):
            I.icd2s_step(st, lp, t)
            F, sc = I.icd2s_get_features(st, lp.z, n)
            assert np.array_equal(F.view(np.uint32), r["F"].view(np.uint32)), t
            assert np.array_equal(sc.view(np.uint32), r["score"].view(np.uint32)), t
            s64 = M.forward(Wb, F.reshape(-1, 6))[0].reshape(lp.z, n)
            assert np.max(np.abs(sc - s64)) <= 1e-3
            assert np.array_equal(I.icd2s_get_hits(st, lp.z, n), r["H"]), t
            x, g, E = I.icd2s_get_state(st, lp.z, n)
            assert np.array_equal(x, r["S"]) and np.array_equal(E, r["E"]), t
            bx, bE = I.icd2s_get_best(st, n)
            assert bE == r["best_E"] and np.array_equal(bx, r["best_x"]), t
    finally:
        I.icd2s_state_destroy(st)
        I.icd2s_qubo_destroy(q)
        I.icd2s_mlp_destroy(m)


@pytest.mark.parametrize("graph", [0, 1])
def test_learned_run_and_log_equal_oracle(L, orc, graph):
    """A whole learned run (state_run, plain or CUDA-graph replay) with the
    improvement log on: trajectory, best solution and every stored log entry
    equal the oracle's; a capacity of 3 exercises the ring buffer."""
    n, seed, iters = 130, 9, 14
    Q = make_qubo(n, 0.7, 12)
    lp = lib_params(I, n, z=4, K=1, m_min=16, m_max=16, m_init=16, alpha=n, c=2, sweeps=24, T_max=300.0,
                    mut_mode=0, patience=0, max_iters=iters, select_mode=1, use_graph=graph)
    op = orc_params(orc, lp)
    m, Wb = _net(_weights(8))
    steps, log = _oracle_chain(orc, Q, op, seed, iters, W=Wb)
    q = I.icd2s_qubo_create(Q)
    st = I.icd2s_state_create(q, lp.z, seed)
    try:
        I.icd2s_state_set_mlp(st, m)
        I.icd2s_log_enable(st, 3)
        g = I.icd2s_state_run(st, n, lp, trace=not graph, want_S=True)
        assert g["iters"] == iters
        assert g["best_E"] == steps[-1]["best_E"] and np.array_equal(g["best_x"], steps[-1]["best_x"])
        assert np.array_equal(g["S"], steps[-1]["S"])
        if not graph:
            tr = np.stack([np.concatenate([r["trace3"], [r["best_E"]]]) for r in steps])
            assert np.array_equal(g["trace"], tr)
        entries, cap = I.icd2s_log_info(st)
        assert entries == len(log) and cap == 3
        F, y, rep = I.icd2s_log_copy(st, n)
        for e in range(max(0, len(log) - 3), len(log)):
            s = e % 3
            assert np.array_equal(F[s].view(np.uint32), log[e][0].view(np.uint32)), e
            assert np.array_equal(y[s], log[e][1]) and rep[s] == log[e][2], e
    finally:
        I.icd2s_state_destroy(st)
        I.icd2s_qubo_destroy(q)
        I.icd2s_mlp_destroy(m)


def test_plain_run_counts_hits_like_oracle(L, orc):
    n, seed = 96, 4
    Q = make_qubo(n, 0.5, 31)
    lp = lib_params(I, n, z=3, K=3, m_min=5, m_max=11, m_init=12, alpha=n, c=2, sweeps=16, T_max=200.0,
                    mut_mode=1, mut_rate=0.1, patience=0, max_iters=5)
    steps, _ = _oracle_chain(orc, Q, orc_params(orc, lp), seed, 5)
    q = I.icd2s_qubo_create(Q)
    st = I.icd2s_state_create(q, lp.z, seed)
    try:
        I.icd2s_state_run(st, n, lp)
        assert np.array_equal(I.icd2s_get_hits(st, lp.z, n), steps[-1]["H"])
    finally:
        I.icd2s_state_destroy(st)
        I.icd2s_qubo_destroy(q)


def test_scores_match_reference(L, orc):
    rows = 1000 + 37
    F = _features(1, rows)
    m, Wb = _net(_weights(2))
    assert np.array_equal(Wb.view(np.uint32), M.bf16_round(_weights(2)).view(np.uint32))
    out = dev(np.zeros(rows, np.float32))
    I.icd2s_mlp_score(m, dev(F).data_ptr(), rows, out.data_ptr())
    s = out.cpu().numpy()
    I.icd2s_mlp_destroy(m)
    assert np.array_equal(s.view(np.uint32), orc.mlp_score_f32(Wb, F).view(np.uint32))
    assert np.max(np.abs(s - M.forward(Wb, F)[0])) <= 1e-3


def test_gradient_matches_reference(L):
    rows = 900 + 5                              # 8 CTAs of 128 rows, the last one ragged
    F = _features(4, rows)
    yv = (np.random.default_rng(5).uniform(size=rows) < 0.25).astype(np.uint8)
    m, Wb = _net(_weights(6))
    torch = torch_cuda()
    grad = torch.zeros(M.NPAR, dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    Fd, yd = dev(F), dev(yv)
    I.icd2s_mlp_grad(m, Fd.data_ptr(), yd.data_ptr(), rows, 3.0, grad.data_ptr(), loss.data_ptr())
    g = grad.cpu().numpy()
    I.icd2s_mlp_destroy(m)
    L_ref, g_ref = M.loss_and_grad(Wb, F, yv, 3.0)
    assert abs(float(loss.cpu()[0]) - L_ref) <= 1e-5 * (1 + abs(L_ref))
    err = np.abs(g - g_ref)
    assert np.all((err <= 1e-3) | (err <= 1e-2 * np.abs(g_ref)))
    assert np.max(err) <= 1e-4                    # far inside the bound in practice


def test_adam_step_follows_definition(L):
    rows = 300
    F = _features(7, rows)
    yv = (np.random.default_rng(8).uniform(size=rows) < 0.4).astype(np.uint8)
    W0 = _weights(9)
    m, _ = _net(W0)
    torch = torch_cuda()
    grad = torch.zeros(M.NPAR, dtype=torch.float32, device="cuda")
    Fd, yd = dev(F), dev(yv)
    I.icd2s_mlp_grad(m, Fd.data_ptr(), yd.data_ptr(), rows, 1.0, grad.data_ptr(), 0)
    g = grad.cpu().numpy().astype(np.float64)
    I.icd2s_mlp_train(m, Fd.data_ptr(), yd.data_ptr(), rows, steps=1, batch=rows, lr=1e-2)
    master, wb = I.icd2s_mlp_get_weights(m)
    I.icd2s_mlp_destroy(m)
    ref, _, _ = M.adam(W0.astype(np.float64), np.zeros(M.NPAR), np.zeros(M.NPAR), g, 1, lr=1e-2)
    assert np.max(np.abs(master - ref)) <= 1e-6
    assert np.array_equal(wb.view(np.uint32), M.bf16_round(master).view(np.uint32))


def test_training_lowers_the_loss(L):
    """Labels y = [f1 < -0.3] (a negative gain): 400 Adam steps on 256-row
    mini-batches drawn on the device lower the reference loss of the BF16
    network well below its start and below the base rate's entropy."""
    rows = 20000
    F = _features(10, rows)
    yv = (F[:, 1] < -0.3).astype(np.uint8)
    m, Wb0 = _net(_weights(11, 0.2))
    Fd, yd = dev(F), dev(yv)
    losses = I.icd2s_mlp_train(m, Fd.data_ptr(), yd.data_ptr(), rows, steps=400, batch=256, lr=3e-3)
    _, Wb1 = I.icd2s_mlp_get_weights(m)
    I.icd2s_mlp_destroy(m)
    l0, l1 = M.loss(Wb0, F, yv), M.loss(Wb1, F, yv)
    p = yv.mean()
    base = -(p * np.log(p) + (1 - p) * np.log(1 - p))
    assert np.all(np.isfinite(losses))
    assert l1 < 0.5 * l0 and l1 < 0.5 * base
    assert losses[-20:].mean() < 0.5 * losses[:20].mean()


@pytest.mark.parametrize("rows", [905, 128, 5000])
def test_tensor_core_gradient_matches_reference(L, rows):
    """The gradient with its 64-wide contractions on the tensor cores (BF16
    operands, FP32 accumulation) agrees with the double-precision reference
    within 1e-3 absolute or 1e-2 relative, its loss within 2e-3 relative, and
    two evaluations are bit-identical (fixed summation order)."""
    F = _features(4 + rows, rows)
    yv = (np.random.default_rng(5).uniform(size=rows) < 0.25).astype(np.uint8)
    m, Wb = _net(_weights(6))
    I.icd2s_mlp_set_tensor_cores(m, True)
    torch = torch_cuda()
    out = []
    Fd, yd = dev(F), dev(yv)
    for _ in range(2):
        grad = torch.zeros(M.NPAR, dtype=torch.float32, device="cuda")
        loss = torch.zeros(1, dtype=torch.float32, device="cuda")
        I.icd2s_mlp_grad(m, Fd.data_ptr(), yd.data_ptr(), rows, 3.0, grad.data_ptr(), loss.data_ptr())
        out.append((grad.cpu().numpy(), float(loss.cpu()[0])))
    I.icd2s_mlp_destroy(m)
    (g, lval), (g2, lval2) = out
    assert np.array_equal(g.view(np.uint32), g2.view(np.uint32)) and lval == lval2
    L_ref, g_ref = M.loss_and_grad(Wb, F, yv, 3.0)
    assert abs(lval - L_ref) <= 2e-3 * (1 + abs(L_ref))
    err = np.abs(g - g_ref)
    assert np.all((err <= 1e-3) | (err <= 1e-2 * np.abs(g_ref)))


def test_tensor_core_training_lowers_the_loss(L):
    """The training test of the FP32 path, with the gradient on the tensor cores."""
    rows = 20000
    F = _features(10, rows)
    yv = (F[:, 1] < -0.3).astype(np.uint8)
    m, Wb0 = _net(_weights(11, 0.2))
    I.icd2s_mlp_set_tensor_cores(m, True)
    Fd, yd = dev(F), dev(yv)
    losses = I.icd2s_mlp_train(m, Fd.data_ptr(), yd.data_ptr(), rows, steps=400, batch=256, lr=3e-3)
    _, Wb1 = I.icd2s_mlp_get_weights(m)
    I.icd2s_mlp_destroy(m)
    l0, l1 = M.loss(Wb0, F, yv), M.loss(Wb1, F, yv)
    p = yv.mean()
    base = -(p * np.log(p) + (1 - p) * np.log(1 - p))
    assert np.all(np.isfinite(losses))
    assert l1 < 0.5 * l0 and l1 < 0.5 * base
