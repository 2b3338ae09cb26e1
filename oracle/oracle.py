"""ctypes binding of the plain C oracle (``icd2s_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline of ``bench.py`` use it; the product library never imports it.

``build()`` compiles the oracle with gcc (``-O2``, no vector intrinsics, same
source on x86 and Arm) into ``oracle/_build/liboracle_icd2s.so``.  Every
wrapper takes and returns numpy arrays; all integer results are exact.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "icd2s_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle_icd2s.so")
_lock = threading.Lock()
_lib = None

TAG_INIT, TAG_ANNEAL, TAG_MUT, TAG_SIZE = 1, 2, 3, 4


def build(force: bool = False) -> str:
    """Compile the oracle shared library (idempotent).  ICD2S_ORACLE_LIB, when
    set, names an already built library to load instead: the planted-mistake
    test points the oracle's pins at mutated builds this way."""
    override = os.environ.get("ICD2S_ORACLE_LIB")
    if override:
        return override
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off", "-fPIC", "-shared",
                           "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Params(C.Structure):
    """Mirror of ``orc_params`` (the oracle's own parameter block)."""
    _fields_ = [
        ("z", C.c_int32), ("K", C.c_int32), ("m_min", C.c_int32), ("m_max", C.c_int32),
        ("m_init", C.c_int32), ("alpha", C.c_int32), ("c", C.c_int32), ("sweeps", C.c_int32),
        ("T_max", C.c_double), ("T_min", C.c_double),
        ("w1", C.c_int64), ("w2", C.c_int64), ("w3", C.c_int64),
        ("mut_mode", C.c_int32), ("mut_rate", C.c_double),
        ("patience", C.c_int32), ("max_iters", C.c_int32), ("select_mode", C.c_int32), ("im_mode", C.c_int32),
        ("ablation", C.c_int32), ("aspiration", C.c_int32), ("im_order", C.c_int32),
    ]


class Result(C.Structure):
    _fields_ = [("iters", C.c_int32), ("best_E", C.c_int64), ("init_best_E", C.c_int64)]


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            L = _lib
            vp, i32, i64, u32, u64, f64 = C.c_void_p, C.c_int32, C.c_int64, C.c_uint32, C.c_uint64, C.c_double
            sig = {
                "orc_philox4x32_10": (None, [vp, vp, vp]),
                "orc_energy": (i64, [vp, i32, vp]),
                "orc_gains": (None, [vp, i32, vp, vp]),
                "orc_energy_batch": (None, [vp, i32, vp, i32, vp]),
                "orc_beta_table": (None, [i32, f64, f64, vp]),
                "orc_nlog_table": (None, [vp]),
                "orc_mutation_rate": (f64, [i32]),
                "orc_init_solutions": (None, [i32, i32, u64, vp]),
                "orc_tabu": (i64, [vp, i32, vp, i32, i32, vp, vp]),
                "orc_tabu_asp": (i64, [vp, i32, vp, i32, i32, vp, vp, i32, vp]),
                "orc_eta": (None, [vp, i32, vp]),
                "orc_eta_hat": (None, [vp, i32, vp]),
                "orc_gamma": (None, [vp, i32, i32, vp]),
                "orc_delta": (None, [vp, i32, vp]),
                "orc_aggregate": (None, [vp, vp, vp, i32, i64, i64, i64, vp]),
                "orc_rank": (None, [vp, i32, vp]),
                "orc_select": (None, [vp, i32, vp, i32, vp]),
                "orc_subqubo_sizes": (None, [i32, i32, i32, u64, u32, u32, vp]),
                "orc_subqubo": (None, [vp, i32, vp, vp, i32, vp, vp]),
                "orc_subqubo_energy": (i64, [vp, i32, vp]),
                "orc_exact_subqubo": (i64, [vp, i32, vp]),
                "orc_anneal": (i64, [vp, i32, vp, i32, vp, vp, u64, u32, u32, vp]),
                "orc_mutate": (i32, [vp, i32, vp, i32, u64, u32, u32, vp]),
                "orc_run": (i32, [vp, i32, C.POINTER(Params), u64, vp, vp, vp, vp, C.POINTER(Result)]),
                "orc_step": (i32, [vp, i32, C.POINTER(Params), u64, i32] + [vp] * 14),
                "orc_features": (None, [i32, vp, vp, vp, vp, vp, vp, i32, i32, i32, vp]),
                "orc_mlp_score_f32": (C.c_float, [vp, vp]),
                "orc_score_key": (i32, [C.c_float]),
                "orc_initial_pass": (None, [vp, i32, C.POINTER(Params), u64, vp, vp]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
        return _lib


def _q(Q):
    Q = np.ascontiguousarray(Q, dtype=np.int8)
    assert Q.ndim == 2 and Q.shape[0] == Q.shape[1]
    return Q, Q.shape[0]


def _u8(x):
    return np.ascontiguousarray(x, dtype=np.uint8)


def _i32(x):
    return np.ascontiguousarray(x, dtype=np.int32)


# --------------------------------------------------------------------------- primitives
def philox(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def energy(Q, x) -> int:
    Q, n = _q(Q)
    x = _u8(x)
    return int(lib().orc_energy(_p(Q), n, _p(x)))


def energy_batch(Q, X):
    Q, n = _q(Q)
    X = _u8(X).reshape(-1, n)
    E = np.zeros(X.shape[0], dtype=np.int64)
    lib().orc_energy_batch(_p(Q), n, _p(X), X.shape[0], _p(E))
    return E


def gains(Q, x):
    Q, n = _q(Q)
    x = _u8(x)
    g = np.zeros(n, dtype=np.int32)
    lib().orc_gains(_p(Q), n, _p(x), _p(g))
    return g


def beta_table(sweeps, T_max, T_min):
    b = np.zeros(max(sweeps, 1), dtype=np.uint32)
    lib().orc_beta_table(sweeps, float(T_max), float(T_min), _p(b))
    return b[:sweeps]


def nlog_table():
    t = np.zeros(4096, dtype=np.uint32)
    lib().orc_nlog_table(_p(t))
    return t


def mutation_rate(t) -> float:
    return float(lib().orc_mutation_rate(int(t)))


def init_solutions(n, z, seed):
    S = np.zeros((z, n), dtype=np.uint8)
    lib().orc_init_solutions(n, z, seed, _p(S))
    return S


def tabu(Q, x, alpha, c):
    """Returns (x_min, E_min, T, C) -- x is not modified."""
    Q, n = _q(Q)
    x = _u8(x).copy()
    T = np.zeros(n, dtype=np.int32)
    Cm = np.zeros(n, dtype=np.int32)
    E = lib().orc_tabu(_p(Q), n, _p(x), alpha, c, _p(T), _p(Cm))
    return x, int(E), T, Cm


def tabu_asp(Q, x, alpha, c, aspiration=True):
    """Tabu search with the aspiration criterion.  Returns (x_min, E_min, T, C, moves)."""
    Q, n = _q(Q)
    x = _u8(x).copy()
    T = np.zeros(n, dtype=np.int32)
    Cm = np.zeros(n, dtype=np.int32)
    mv = np.zeros(max(alpha, 1), dtype=np.int32)
    E = lib().orc_tabu_asp(_p(Q), n, _p(x), alpha, c, _p(T), _p(Cm), 1 if aspiration else 0, _p(mv))
    return x, int(E), T, Cm, mv[:alpha]


def eta(Q):
    Q, n = _q(Q)
    e = np.zeros(n, dtype=np.int64)
    lib().orc_eta(_p(Q), n, _p(e))
    return e


def eta_hat(eta_v):
    e = np.ascontiguousarray(eta_v, dtype=np.int64)
    out = np.zeros(e.shape[0], dtype=np.int32)
    lib().orc_eta_hat(_p(e), e.shape[0], _p(out))
    return out


def gamma(S):
    S = _u8(S)
    z, n = S.shape
    out = np.zeros(n, dtype=np.int32)
    lib().orc_gamma(_p(S), z, n, _p(out))
    return out


def delta(T):
    T = _i32(T)
    out = np.zeros(T.shape[0], dtype=np.int32)
    lib().orc_delta(_p(T), T.shape[0], _p(out))
    return out


W_DEFAULT = (65536, 65536, 32768)


def aggregate(eta_hat_v, gamma_v, delta_v, w=W_DEFAULT):
    eh, g, d = _i32(eta_hat_v), _i32(gamma_v), _i32(delta_v)
    n = eh.shape[0]
    A = np.zeros(n, dtype=np.int32)
    lib().orc_aggregate(_p(eh), _p(g), _p(d), n, int(w[0]), int(w[1]), int(w[2]), _p(A))
    return A


def rank(key):
    k = _i32(key)
    order = np.zeros(k.shape[0], dtype=np.int32)
    lib().orc_rank(_p(k), k.shape[0], _p(order))
    return order


def select(A, sizes):
    A = _i32(A)
    sizes = _i32(sizes)
    idx = np.zeros(int(sizes.sum()), dtype=np.int32)
    lib().orc_select(_p(A), A.shape[0], _p(sizes), sizes.shape[0], _p(idx))
    return idx


def subqubo_sizes(K, m_min, m_max, seed, p, it):
    s = np.zeros(K, dtype=np.int32)
    lib().orc_subqubo_sizes(K, m_min, m_max, seed, p, it, _p(s))
    return s


def subqubo(Q, x, S):
    """Eq. 4: (Q' with bias on the diagonal [m, m] int32, b [m] int64)."""
    Q, n = _q(Q)
    x = _u8(x)
    S = _i32(S)
    m = S.shape[0]
    Qs = np.zeros((m, m), dtype=np.int32)
    b = np.zeros(m, dtype=np.int64)
    lib().orc_subqubo(_p(Q), n, _p(x), _p(S), m, _p(Qs), _p(b))
    return Qs, b


def subqubo_energy(Qs, xs) -> int:
    Qs = _i32(Qs)
    xs = _u8(xs)
    return int(lib().orc_subqubo_energy(_p(Qs), Qs.shape[0], _p(xs)))


def exact_subqubo(Qs, xs):
    """Exact minimiser of the subQUBO objective (ties: smallest sum y_a 2^a).
    Returns (y, f(y) - f(xs))."""
    Qs = np.ascontiguousarray(Qs, dtype=np.int32)
    m = Qs.shape[0]
    y = _u8(xs).copy()
    dE = lib().orc_exact_subqubo(_p(Qs), m, _p(y))
    return y, int(dE)


def anneal(Qs, xs, beta, nlog, seed, slot, it):
    """Returns (xs_after, dE, accepts)."""
    Qs = _i32(Qs)
    xs = _u8(xs).copy()
    b = np.ascontiguousarray(beta, dtype=np.uint32)
    t = np.ascontiguousarray(nlog, dtype=np.uint32)
    acc = np.zeros(1, dtype=np.int64)
    dE = lib().orc_anneal(_p(Qs), Qs.shape[0], _p(xs), b.shape[0], _p(b), _p(t), seed,
                          slot, it, _p(acc))
    return xs, int(dE), int(acc[0])


def mutate(A, in_sel, L, seed, p, it, x):
    """Returns (x_after, flips)."""
    A = _i32(A)
    sel = _u8(in_sel)
    x = _u8(x).copy()
    f = lib().orc_mutate(_p(A), A.shape[0], _p(sel), L, seed, p, it, _p(x))
    return x, int(f)


def default_params(n, **kw) -> Params:
    """Table 1 defaults (z = 4, c = n/150, alpha = 5n, w = (1, 1, 0.5)) with
    c clamped to [2, n] (reading S5) and an IM of size 50 (Section 4.1)."""
    m = kw.pop("m", min(50, n))
    P = Params(z=4, K=1, m_min=m, m_max=m, m_init=m, alpha=5 * n,
               c=max(2, min(n, n // 150)), sweeps=256, T_max=100.0, T_min=1.0,
               w1=65536, w2=65536, w3=32768, mut_mode=0, mut_rate=0.0,
               patience=30, max_iters=100)
    for k, v in kw.items():
        setattr(P, k, v)
    return P


def run(Q, prm: Params, seed: int, trace: bool = True):
    """Algorithm 2.  Returns dict(best_x, best_E, S, trace[iters, 3z+1], init_E, iters)."""
    Q, n = _q(Q)
    z = prm.z
    best_x = np.zeros(n, dtype=np.uint8)
    S = np.zeros((z, n), dtype=np.uint8)
    tr = np.zeros((max(prm.max_iters, 1), 3 * z + 1), dtype=np.int64) if trace else None
    init_E = np.zeros(z, dtype=np.int64)
    res = Result()
    it = lib().orc_run(_p(Q), n, C.byref(prm), seed, _p(best_x), _p(S),
                       _p(tr) if tr is not None else None, _p(init_E), C.byref(res))
    return dict(best_x=best_x, best_E=int(res.best_E), S=S,
                trace=tr[:it] if tr is not None else None, init_E=init_E,
                init_best_E=int(res.init_best_E), iters=int(it))


def step(Q, prm: Params, seed: int, t: int, S, best_E=None, best_x=None, H=None, W=None, want_features=False):
    """One outer iteration of Algorithm 2 from the solution set S (not
    modified).  Returns dict(S, E, trace3, best_E, best_x, T, A, C, H,
    improved, winner, F, score): T/C the Tabu toggle counts and final tabu
    memory of each replica, H the per-replica selection hit counts (H input
    + 1 for every variable placed in a subQUBO this iteration), winner the
    replica last copied into best_x (-1: none).  W (4673 BF16-valued floats)
    is the proposal network, required when prm.select_mode != 0; with
    want_features, F [z][n][6] and (when W is given) score [z][n] are the
    features and scores at selection time."""
    Q, n = _q(Q)
    S = _u8(S).copy()
    z = prm.z
    assert S.shape == (z, n)
    eh = eta_hat(eta(Q))
    E = np.zeros(z, np.int64)
    tr = np.zeros(3 * z, np.int64)
    bE = np.array([np.iinfo(np.int64).max if best_E is None else best_E], np.int64)
    bx = np.zeros(n, np.uint8) if best_x is None else _u8(best_x).copy()
    T = np.zeros((z, n), np.int32)
    A = np.zeros((z, n), np.int32)
    Cm = np.zeros((z, n), np.int32)
    Hm = np.zeros((z, n), np.int32) if H is None else np.ascontiguousarray(H, np.int32).copy()
    assert Hm.shape == (z, n)
    Wf = None if W is None else np.ascontiguousarray(W, np.float32)
    assert Wf is None or Wf.shape == (NPAR,)
    assert prm.select_mode == 0 or Wf is not None
    F = np.zeros((z, n, 6), np.float32) if want_features else None
    sc = np.zeros((z, n), np.float32) if (want_features and Wf is not None) else None
    win = np.zeros(1, np.int32)
    nul = C.c_void_p(None)
    imp = lib().orc_step(_p(Q), n, C.byref(prm), seed, t, _p(eh), _p(S), _p(E), _p(tr), _p(bE), _p(bx),
                         _p(T), _p(A), _p(Cm), _p(Hm), nul if Wf is None else _p(Wf),
                         nul if F is None else _p(F), nul if sc is None else _p(sc), _p(win))
    assert imp >= 0
    return dict(S=S, E=E, trace3=tr, best_E=int(bE[0]), best_x=bx, T=T, A=A, C=Cm, H=Hm, improved=int(imp),
                winner=int(win[0]), F=F, score=sc)


# --------------------------------------------------------------------------- learned selection
NPAR = 4673  # 6-64-64-1 network: W1[64][6], b1[64], W2[64][64], b2[64], w3[64], b3


def features(x, g, T, Cm, H, eta_hat_v, t, alpha, c):
    """Per-variable features of one solution at selection time, float32 [n][6]."""
    x, g, T, Cm, H, eh = _u8(x), _i32(g), _i32(T), _i32(Cm), _i32(H), _i32(eta_hat_v)
    n = x.shape[0]
    F = np.zeros((n, 6), np.float32)
    lib().orc_features(n, _p(x), _p(g), _p(T), _p(Cm), _p(H), _p(eh), int(t), int(alpha), int(c), _p(F))
    return F


def mlp_score_f32(W, F):
    """Float scores of the rows of F [rows][6] (fused multiply-adds in a fixed order)."""
    Wf = np.ascontiguousarray(W, np.float32)
    F = np.ascontiguousarray(F, np.float32).reshape(-1, 6)
    out = np.zeros(F.shape[0], np.float32)
    for r in range(F.shape[0]):
        out[r] = lib().orc_mlp_score_f32(_p(Wf), _p(F[r]))
    return out


def score_key(s) -> int:
    return int(lib().orc_score_key(float(np.float32(s))))


def initial_pass(Q, prm: Params, seed: int, S):
    """Call_IM_Solution_Set on S (not modified).  Returns (S_after, E)."""
    Q, n = _q(Q)
    S = _u8(S).copy()
    E = np.zeros(prm.z, np.int64)
    lib().orc_initial_pass(_p(Q), n, C.byref(prm), seed, _p(S), _p(E))
    return S, E
