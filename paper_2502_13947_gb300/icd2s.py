"""Thin ctypes binding of ``libicd2s.so`` (declared in ``include/icd2s.h``).

Argument marshalling only: every step runs in the library's CUDA kernels.
Each ``icd2s_*`` function here calls the C entry point of the same name and
raises ``ICD2SError`` on a non-zero status.  Device buffers are passed as raw
addresses (e.g. ``torch.Tensor.data_ptr()``), streams as ``cudaStream_t``
integers (e.g. ``torch.cuda.current_stream().cuda_stream``) or 0.

There is no CPU fallback: if the shared library is missing the first call
raises, naming the build step (``python -m paper_2502_13947_gb300.build``).
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libicd2s.so")

OK, ERR_ARG, ERR_ASYMMETRIC, ERR_RANGE, ERR_OOM, ERR_CUDA, ERR_TIMEOUT, ERR_INVARIANT, ERR_STATE = (
    0, -1, -2, -3, -4, -5, -6, -7, -8)

# every entry point declared in include/icd2s.h
EXPORTS = (
    "icd2s_last_error", "icd2s_version", "icd2s_default_params", "icd2s_qubo_create", "icd2s_qubo_destroy",
    "icd2s_qubo_size", "icd2s_qubo_gain_bound", "icd2s_energy", "icd2s_state_create", "icd2s_state_destroy", "icd2s_state_load",
    "icd2s_get_state", "icd2s_get_best", "icd2s_tabu", "icd2s_get_tabu", "icd2s_select_subqubos",
    "icd2s_get_control", "icd2s_anneal_subqubos_batch", "icd2s_apply_flips_update_gains", "icd2s_mutate",
    "icd2s_best_update", "icd2s_initial_pass", "icd2s_step", "icd2s_step_host", "icd2s_run", "icd2s_tables",
    "icd2s_set_timing", "icd2s_get_phase_ms", "icd2s_kernel_launches", "icd2s_apply_flips_static",
    "icd2s_set_tuning", "icd2s_get_tuning", "icd2s_autotune", "icd2s_refresh", "icd2s_get_refresh_ms",
    "icd2s_state_run", "icd2s_mlp_create", "icd2s_mlp_destroy", "icd2s_mlp_set_weights", "icd2s_mlp_get_weights",
    "icd2s_mlp_score", "icd2s_mlp_grad", "icd2s_mlp_train", "icd2s_state_set_mlp", "icd2s_get_features",
    "icd2s_get_hits", "icd2s_log_enable", "icd2s_log_info", "icd2s_log_copy", "icd2s_get_apply_ms",
    "icd2s_exact_subqubos_batch", "icd2s_tabu_aspiration", "icd2s_state_save", "icd2s_checkpoint_info",
    "icd2s_state_restore", "icd2s_debug_fail_allocations_after", "icd2s_state_create_shard",
    "icd2s_step_shard_begin", "icd2s_step_shard_finish", "icd2s_get_best_info", "icd2s_debug_refresh_stall",
    "icd2s_im_round", "icd2s_mlp_set_tensor_cores",
)
MLP_PARAMS = 4673
PHASES = ("tabu", "select", "anneal", "apply_anneal", "mutate", "apply_mutate", "best")


class ICD2SError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("icd2s error %d: %s" % (code, msg))
        self.code = code


class Params(C.Structure):
    _fields_ = [
        ("z", C.c_int32), ("K", C.c_int32), ("m_min", C.c_int32), ("m_max", C.c_int32), ("m_init", C.c_int32),
        ("alpha", C.c_int32), ("c", C.c_int32), ("sweeps", C.c_int32), ("T_max", C.c_double), ("T_min", C.c_double),
        ("w1", C.c_int64), ("w2", C.c_int64), ("w3", C.c_int64), ("mut_mode", C.c_int32), ("mut_rate", C.c_double),
        ("patience", C.c_int32), ("max_iters", C.c_int32), ("use_graph", C.c_int32), ("refresh_every", C.c_int32),
        ("select_mode", C.c_int32), ("stop_at_target", C.c_int32), ("target_E", C.c_int64),
        ("im_mode", C.c_int32), ("ablation", C.c_int32), ("aspiration", C.c_int32), ("im_order", C.c_int32),
        ("t_start", C.c_int32), ("reserved", C.c_int32 * 1),
    ]


class AnnealParams(C.Structure):
    _fields_ = [("sweeps", C.c_int32), ("T_max", C.c_double), ("T_min", C.c_double), ("iter", C.c_uint32),
                ("per_replica", C.c_int32)]


class SelectParams(C.Structure):
    _fields_ = [("w1", C.c_int64), ("w2", C.c_int64), ("w3", C.c_int64), ("K", C.c_int32), ("m_min", C.c_int32),
                ("m_max", C.c_int32), ("iter", C.c_uint32)]


class MutateParams(C.Structure):
    _fields_ = [("mut_mode", C.c_int32), ("mut_rate", C.c_double), ("iter", C.c_uint32)]


class Stats(C.Structure):
    _fields_ = [("iters", C.c_int32), ("best_E", C.c_int64), ("init_best_E", C.c_int64),
                ("anneal_attempts", C.c_int64), ("tabu_moves", C.c_int64), ("device_ms", C.c_double),
                ("ttt_ms", C.c_double), ("hit_iter", C.c_int32)]


class TrainParams(C.Structure):
    _fields_ = [("steps", C.c_int32), ("batch", C.c_int32), ("lr", C.c_float), ("beta1", C.c_float),
                ("beta2", C.c_float), ("eps", C.c_float), ("pos_weight", C.c_float), ("reserved", C.c_int32 * 3)]


_lock = threading.Lock()
_lib = None


def lib():
    """Loads the library (once).  Raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ICD2SError(ERR_STATE, "%s is missing: build it with `python -m paper_2502_13947_gb300.build` "
                                            "(or __graft_entry__.build())" % LIB_PATH)
            L = C.CDLL(LIB_PATH)
            vp, i32, i64, u32, u64, f64 = C.c_void_p, C.c_int32, C.c_int64, C.c_uint32, C.c_uint64, C.c_double
            P = C.POINTER
            sig = {
                "icd2s_last_error": (C.c_char_p, []),
                "icd2s_version": (i32, []),
                "icd2s_default_params": (C.c_int, [i32, P(Params)]),
                "icd2s_qubo_create": (C.c_int, [vp, i32, P(vp)]),
                "icd2s_qubo_destroy": (C.c_int, [vp]),
                "icd2s_qubo_size": (C.c_int, [vp, P(i32)]),
                "icd2s_qubo_gain_bound": (C.c_int, [vp, P(C.c_int64)]),
                "icd2s_energy": (C.c_int, [vp, vp, i32, vp, vp]),
                "icd2s_state_create": (C.c_int, [vp, i32, u64, P(vp)]),
                "icd2s_state_create_shard": (C.c_int, [vp, i32, i32, i32, u64, P(vp)]),
                "icd2s_step_shard_begin": (C.c_int, [vp, P(Params), i32, vp, vp]),
                "icd2s_step_shard_finish": (C.c_int, [vp, P(Params), i32, vp, vp]),
                "icd2s_get_best_info": (C.c_int, [vp, P(C.c_int64), P(i32), P(i32)]),
                "icd2s_debug_refresh_stall": (C.c_int, [vp, i32, i32]),
                "icd2s_im_round": (C.c_int, [vp, P(Params), i32, vp]),
                "icd2s_mlp_set_tensor_cores": (C.c_int, [vp, i32]),
                "icd2s_state_destroy": (C.c_int, [vp]),
                "icd2s_state_load": (C.c_int, [vp, vp, i32, vp]),
                "icd2s_get_state": (C.c_int, [vp, vp, vp, vp]),
                "icd2s_get_best": (C.c_int, [vp, vp, vp]),
                "icd2s_state_save": (C.c_int, [vp, i32, vp, C.c_size_t, P(C.c_size_t)]),
                "icd2s_checkpoint_info": (C.c_int, [vp, C.c_size_t, P(i32), P(i32), P(i32), P(u64)]),
                "icd2s_state_restore": (C.c_int, [vp, vp, C.c_size_t, P(i32)]),
                "icd2s_tabu": (C.c_int, [vp, i32, i32, vp]),
                "icd2s_get_tabu": (C.c_int, [vp, vp, vp]),
                "icd2s_select_subqubos": (C.c_int, [vp, P(SelectParams), vp, vp, vp]),
                "icd2s_get_control": (C.c_int, [vp, vp, vp, vp]),
                "icd2s_anneal_subqubos_batch": (C.c_int, [vp, vp, vp, i32, P(AnnealParams), vp, vp, vp]),
                "icd2s_apply_flips_update_gains": (C.c_int, [vp, vp, vp]),
                "icd2s_mutate": (C.c_int, [vp, P(MutateParams), vp, vp]),
                "icd2s_best_update": (C.c_int, [vp, vp]),
                "icd2s_initial_pass": (C.c_int, [vp, P(Params), vp]),
                "icd2s_step": (C.c_int, [vp, P(Params), i32, vp]),
                "icd2s_step_host": (C.c_int, [vp, P(Params), i32, vp, vp, vp, vp]),
                "icd2s_run": (C.c_int, [vp, P(Params), u64, vp, vp, P(Stats), vp, vp]),
                "icd2s_tables": (C.c_int, [i32, f64, f64, vp, vp]),
                "icd2s_set_timing": (C.c_int, [vp, i32]),
                "icd2s_get_phase_ms": (C.c_int, [vp, vp]),
                "icd2s_kernel_launches": (C.c_int, [P(u64)]),
                "icd2s_debug_fail_allocations_after": (C.c_int, [i32]),
                "icd2s_apply_flips_static": (C.c_int, [vp, i32, i32, i32, vp, vp, vp, vp, vp]),
                "icd2s_set_tuning": (C.c_int, [vp, vp]),
                "icd2s_get_tuning": (C.c_int, [vp, vp]),
                "icd2s_autotune": (C.c_int, [vp, P(Params), vp, vp]),
                "icd2s_refresh": (C.c_int, [vp, i32, P(i32), vp]),
                "icd2s_get_refresh_ms": (C.c_int, [vp, P(f64)]),
                "icd2s_get_apply_ms": (C.c_int, [vp, P(f64)]),
                "icd2s_exact_subqubos_batch": (C.c_int, [vp, vp, vp, i32, i32, vp, vp, vp]),
                "icd2s_tabu_aspiration": (C.c_int, [vp, i32, i32, vp]),
                "icd2s_state_run": (C.c_int, [vp, P(Params), vp, vp, P(Stats), vp, vp]),
                "icd2s_mlp_create": (C.c_int, [u64, P(vp)]),
                "icd2s_mlp_destroy": (C.c_int, [vp]),
                "icd2s_mlp_set_weights": (C.c_int, [vp, vp]),
                "icd2s_mlp_get_weights": (C.c_int, [vp, vp, vp]),
                "icd2s_mlp_score": (C.c_int, [vp, vp, i64, vp, vp]),
                "icd2s_mlp_grad": (C.c_int, [vp, vp, vp, i64, C.c_float, vp, vp, vp]),
                "icd2s_mlp_train": (C.c_int, [vp, vp, vp, i64, P(TrainParams), vp, vp]),
                "icd2s_state_set_mlp": (C.c_int, [vp, vp]),
                "icd2s_get_features": (C.c_int, [vp, vp, vp]),
                "icd2s_get_hits": (C.c_int, [vp, vp]),
                "icd2s_log_enable": (C.c_int, [vp, i32]),
                "icd2s_log_info": (C.c_int, [vp, P(i32), P(i32)]),
                "icd2s_log_copy": (C.c_int, [vp, vp, vp, vp, i32, vp]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
        return _lib


def _check(rc):
    if rc != OK:
        raise ICD2SError(rc, lib().icd2s_last_error().decode(errors="replace"))


def _np(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def _s(stream):
    return C.c_void_p(int(stream) if stream else 0)


# --------------------------------------------------------------------------- entry points
def icd2s_version() -> int:
    return int(lib().icd2s_version())


def icd2s_default_params(n: int, **overrides) -> Params:
    p = Params()
    _check(lib().icd2s_default_params(n, C.byref(p)))
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def icd2s_qubo_create(Q: np.ndarray) -> C.c_void_p:
    Q = np.ascontiguousarray(Q, dtype=np.int8)
    if Q.ndim != 2 or Q.shape[0] != Q.shape[1]:
        raise ValueError("Q must be square")
    h = C.c_void_p()
    _check(lib().icd2s_qubo_create(_np(Q), Q.shape[0], C.byref(h)))
    return h


def icd2s_qubo_destroy(h) -> None:
    _check(lib().icd2s_qubo_destroy(h))


def icd2s_qubo_size(h) -> int:
    n = C.c_int32()
    _check(lib().icd2s_qubo_size(h, C.byref(n)))
    return n.value


def icd2s_qubo_gain_bound(h) -> int:
    b = C.c_int64()
    _check(lib().icd2s_qubo_gain_bound(h, C.byref(b)))
    return b.value


def icd2s_energy(q, x_dev: int, count: int, E_dev: int, stream=0) -> None:
    _check(lib().icd2s_energy(q, C.c_void_p(x_dev), count, C.c_void_p(E_dev), _s(stream)))


def icd2s_state_create(q, replicas: int, seed: int) -> C.c_void_p:
    h = C.c_void_p()
    _check(lib().icd2s_state_create(q, replicas, C.c_uint64(seed), C.byref(h)))
    return h


def icd2s_state_destroy(st) -> None:
    _check(lib().icd2s_state_destroy(st))


def icd2s_state_load(st, x, x_is_device: bool = False, stream=0) -> None:
    if x_is_device:
        _check(lib().icd2s_state_load(st, C.c_void_p(int(x)), 1, _s(stream)))
    else:
        x = np.ascontiguousarray(x, dtype=np.uint8)
        _check(lib().icd2s_state_load(st, _np(x), 0, _s(stream)))


def icd2s_get_state(st, R: int, n: int, x=None, E=None, want_g: bool = True):
    """Host copies of the solutions, gains and energies (x / E may be given:
    uint8 [R][n] / int64 [R] arrays, e.g. pinned; want_g=False skips g)."""
    x = np.zeros((R, n), np.uint8) if x is None else x
    g = np.zeros((R, n), np.int32) if want_g else None
    E = np.zeros(R, np.int64) if E is None else E
    _check(lib().icd2s_get_state(st, _np(x), _np(g), _np(E)))
    return x, g, E


def icd2s_get_best(st, n: int):
    x = np.zeros(n, np.uint8)
    E = np.zeros(1, np.int64)
    _check(lib().icd2s_get_best(st, _np(x), _np(E)))
    return x, int(E[0])


def icd2s_get_best_info(st):
    """(best energy, its global replica index, the stamp of the update that set it)."""
    E, r, t = C.c_int64(), C.c_int32(), C.c_int32()
    _check(lib().icd2s_get_best_info(st, C.byref(E), C.byref(r), C.byref(t)))
    return int(E.value), int(r.value), int(t.value)


def icd2s_state_create_shard(q, replicas: int, replica_base: int, replicas_total: int, seed: int) -> C.c_void_p:
    """Replicas replica_base .. replica_base + replicas - 1 of a set of replicas_total."""
    h = C.c_void_p()
    _check(lib().icd2s_state_create_shard(q, replicas, replica_base, replicas_total, C.c_uint64(seed),
                                          C.byref(h)))
    return h


def icd2s_state_save(st, t_next: int) -> bytes:
    """The state's checkpoint (see include/icd2s.h for the format)."""
    size = C.c_size_t()
    _check(lib().icd2s_state_save(st, t_next, None, 0, C.byref(size)))
    buf = C.create_string_buffer(size.value)
    _check(lib().icd2s_state_save(st, t_next, buf, size.value, C.byref(size)))
    return buf.raw[:size.value]


def icd2s_checkpoint_info(blob: bytes):
    """(n, replicas, t_next, seed) of a checkpoint; raises on a bad one."""
    n, R, t = C.c_int32(), C.c_int32(), C.c_int32()
    seed = C.c_uint64()
    _check(lib().icd2s_checkpoint_info(blob, len(blob), C.byref(n), C.byref(R), C.byref(t), C.byref(seed)))
    return n.value, R.value, t.value, seed.value


def icd2s_state_restore(st, blob: bytes) -> int:
    """Restores a checkpoint into st; returns the iteration to continue with."""
    t = C.c_int32()
    _check(lib().icd2s_state_restore(st, blob, len(blob), C.byref(t)))
    return t.value


def icd2s_debug_fail_allocations_after(count: int) -> None:
    """Testing aid: every device allocation after the next `count` fails
    (ICD2S_ERR_OOM) until count < 0 switches the hook off."""
    _check(lib().icd2s_debug_fail_allocations_after(count))


def icd2s_tabu(st, alpha: int, c: int, stream=0) -> None:
    _check(lib().icd2s_tabu(st, alpha, c, _s(stream)))


def icd2s_tabu_aspiration(st, alpha: int, c: int, stream=0) -> None:
    _check(lib().icd2s_tabu_aspiration(st, alpha, c, _s(stream)))


def icd2s_get_tabu(st, R: int, n: int):
    T = np.zeros((R, n), np.int32)
    Cm = np.zeros((R, n), np.int32)
    _check(lib().icd2s_get_tabu(st, _np(T), _np(Cm)))
    return T, Cm


def icd2s_select_subqubos(st, sp: SelectParams, idx_dev: int, off_dev: int, stream=0) -> None:
    _check(lib().icd2s_select_subqubos(st, C.byref(sp), C.c_void_p(idx_dev), C.c_void_p(off_dev), _s(stream)))


def icd2s_get_control(st, R: int, n: int):
    A = np.zeros((R, n), np.int32)
    gam = np.zeros(n, np.int32)
    dl = np.zeros((R, n), np.int32)
    _check(lib().icd2s_get_control(st, _np(A), _np(gam), _np(dl)))
    return A, gam, dl


def icd2s_anneal_subqubos_batch(st, idx_dev: int, off_dev: int, count: int, ap: AnnealParams, flips_dev: int,
                                dE_dev: int = 0, stream=0) -> None:
    _check(lib().icd2s_anneal_subqubos_batch(st, C.c_void_p(idx_dev), C.c_void_p(off_dev), count, C.byref(ap),
                                             C.c_void_p(flips_dev), C.c_void_p(dE_dev or None), _s(stream)))


def icd2s_exact_subqubos_batch(st, idx_dev: int, off_dev: int, count: int, per_replica: int, flips_dev: int,
                               dE_dev: int = 0, stream=0) -> None:
    _check(lib().icd2s_exact_subqubos_batch(st, idx_dev, off_dev, count, per_replica, flips_dev, dE_dev or None,
                                            _s(stream)))


def icd2s_apply_flips_update_gains(st, flips_dev: int, stream=0) -> None:
    _check(lib().icd2s_apply_flips_update_gains(st, C.c_void_p(flips_dev), _s(stream)))


def icd2s_mutate(st, mp: MutateParams, flips_dev: int = 0, stream=0) -> None:
    _check(lib().icd2s_mutate(st, C.byref(mp), C.c_void_p(flips_dev or None), _s(stream)))


def icd2s_best_update(st, stream=0) -> None:
    _check(lib().icd2s_best_update(st, _s(stream)))


def icd2s_initial_pass(st, p: Params, stream=0) -> None:
    _check(lib().icd2s_initial_pass(st, C.byref(p), _s(stream)))


def icd2s_step(st, p: Params, t: int, stream=0) -> None:
    _check(lib().icd2s_step(st, C.byref(p), t, _s(stream)))


def icd2s_im_round(st, p: Params, t: int, stream=0) -> None:
    """One Ising-machine round: selection, batched anneal, write-back (no Tabu, no mutation)."""
    _check(lib().icd2s_im_round(st, C.byref(p), t, _s(stream)))


def icd2s_step_shard_begin(st, p: Params, t: int, counts_dev: int, stream=0) -> None:
    """First half of iteration t on a replica shard; writes its column counts (int32 [n], device)."""
    _check(lib().icd2s_step_shard_begin(st, C.byref(p), t, C.c_void_p(counts_dev), _s(stream)))


def icd2s_step_shard_finish(st, p: Params, t: int, counts_dev: int, stream=0) -> None:
    """Rest of iteration t, with gamma from the column counts of every shard (int32 [n], device)."""
    _check(lib().icd2s_step_shard_finish(st, C.byref(p), t, C.c_void_p(counts_dev), _s(stream)))


def icd2s_step_host(st, p: Params, t: int, x_in=None, x_out=None, E_out=None, stream=0) -> None:
    """Host-buffer step.  x_in / x_out / E_out are numpy arrays (pinned memory
    may be passed as numpy views of pinned torch tensors) or None."""
    _check(lib().icd2s_step_host(st, C.byref(p), t, _np(x_in), _np(x_out), _np(E_out), _s(stream)))


def _run_out(st, x, E, tr, S, trace, want_S):
    out = dict(best_x=x, best_E=int(E[0]), iters=st.iters, init_best_E=st.init_best_E,
               anneal_attempts=st.anneal_attempts, tabu_moves=st.tabu_moves, device_ms=st.device_ms,
               ttt_ms=st.ttt_ms, hit_iter=st.hit_iter)
    if trace:
        out["trace"] = tr[:st.iters]
    if want_S:
        out["S"] = S
    return out


def icd2s_run(q, p: Params, seed: int, trace: bool = False, want_S: bool = False):
    n = icd2s_qubo_size(q)
    x = np.zeros(n, np.uint8)
    E = np.zeros(1, np.int64)
    st = Stats()
    tr = np.zeros((max(p.max_iters, 1), 3 * p.z + 1), np.int64) if trace else None
    S = np.zeros((p.z, n), np.uint8) if want_S else None
    _check(lib().icd2s_run(q, C.byref(p), C.c_uint64(seed), _np(x), _np(E), C.byref(st), _np(tr), _np(S)))
    return _run_out(st, x, E, tr, S, trace, want_S)


def icd2s_state_run(state, n: int, p: Params, trace: bool = False, want_S: bool = False):
    """Algorithm 2 on an existing state (see icd2s_run for the outputs).  With
    p.t_start > 0 (a state restored from a checkpoint) the run continues at
    that iteration and the trace rows before it are left zero."""
    x = np.zeros(n, np.uint8)
    E = np.zeros(1, np.int64)
    st = Stats()
    tr = np.zeros((max(p.max_iters, 1), 3 * p.z + 1), np.int64) if trace else None
    S = np.zeros((p.z, n), np.uint8) if want_S else None
    _check(lib().icd2s_state_run(state, C.byref(p), _np(x), _np(E), C.byref(st), _np(tr), _np(S)))
    return _run_out(st, x, E, tr, S, trace, want_S)


# ----------------------------------------------------------------------------- learned selection
def icd2s_mlp_create(seed: int) -> C.c_void_p:
    h = C.c_void_p()
    _check(lib().icd2s_mlp_create(C.c_uint64(seed), C.byref(h)))
    return h


def icd2s_mlp_destroy(m) -> None:
    _check(lib().icd2s_mlp_destroy(m))


def icd2s_mlp_set_weights(m, W) -> None:
    W = np.ascontiguousarray(W, np.float32)
    assert W.shape == (MLP_PARAMS,)
    _check(lib().icd2s_mlp_set_weights(m, _np(W)))


def icd2s_mlp_get_weights(m):
    """Returns (master float32 [4673], bf16 values as float32 [4673])."""
    a = np.zeros(MLP_PARAMS, np.float32)
    b = np.zeros(MLP_PARAMS, np.float32)
    _check(lib().icd2s_mlp_get_weights(m, _np(a), _np(b)))
    return a, b


def icd2s_mlp_score(m, F_dev: int, rows: int, score_dev: int, stream=0) -> None:
    _check(lib().icd2s_mlp_score(m, F_dev, rows, score_dev, _s(stream)))


def icd2s_mlp_grad(m, F_dev: int, y_dev: int, rows: int, pos_weight: float, grad_dev: int, loss_dev: int,
                   stream=0) -> None:
    _check(lib().icd2s_mlp_grad(m, F_dev, y_dev, rows, pos_weight, grad_dev or None, loss_dev or None, _s(stream)))


def icd2s_mlp_train(m, F_dev: int, y_dev: int, rows: int, steps: int, batch: int, lr: float = 1e-3,
                    beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8, pos_weight: float = 1.0, stream=0):
    """Returns the per-step mean batch losses (numpy float32 [steps])."""
    tp = TrainParams(steps=steps, batch=batch, lr=lr, beta1=beta1, beta2=beta2, eps=eps, pos_weight=pos_weight)
    loss = np.zeros(max(steps, 1), np.float32)
    _check(lib().icd2s_mlp_train(m, F_dev, y_dev, rows, C.byref(tp), _np(loss), _s(stream)))
    return loss[:steps]


def icd2s_state_set_mlp(st, m) -> None:
    _check(lib().icd2s_state_set_mlp(st, m))


def icd2s_get_features(st, R: int, n: int, scores: bool = True):
    F = np.zeros((R, n, 6), np.float32)
    sc = np.zeros((R, n), np.float32) if scores else None
    _check(lib().icd2s_get_features(st, _np(F), _np(sc)))
    return F, sc


def icd2s_get_hits(st, R: int, n: int):
    H = np.zeros((R, n), np.int32)
    _check(lib().icd2s_get_hits(st, _np(H)))
    return H


def icd2s_log_enable(st, capacity: int) -> None:
    _check(lib().icd2s_log_enable(st, capacity))


def icd2s_log_info(st):
    e, c = C.c_int32(0), C.c_int32(0)
    _check(lib().icd2s_log_info(st, C.byref(e), C.byref(c)))
    return int(e.value), int(c.value)


def icd2s_log_copy(st, n: int):
    """Host copies of the stored log entries: (F [cnt][n][6], y [cnt][n], replica [cnt])."""
    e, c = icd2s_log_info(st)
    cnt = min(e, c)
    F = np.zeros((max(cnt, 1), n, 6), np.float32)
    y = np.zeros((max(cnt, 1), n), np.uint8)
    r = np.zeros(max(cnt, 1), np.int32)
    _check(lib().icd2s_log_copy(st, _np(F), _np(y), _np(r), 0, None))
    return F[:cnt], y[:cnt], r[:cnt]


def icd2s_log_copy_device(st, F_dev: int, y_dev: int, replica_dev: int = 0, stream=0) -> None:
    _check(lib().icd2s_log_copy(st, F_dev, y_dev, replica_dev or None, 1, _s(stream)))


def icd2s_tables(sweeps: int, T_max: float, T_min: float):
    b = np.zeros(max(sweeps, 1), np.uint32)
    t = np.zeros(4096, np.uint32)
    _check(lib().icd2s_tables(sweeps, T_max, T_min, _np(b), _np(t)))
    return b[:sweeps], t


def icd2s_set_timing(st, enable: bool = True) -> None:
    _check(lib().icd2s_set_timing(st, 1 if enable else 0))


def icd2s_get_phase_ms(st) -> dict:
    ms = np.zeros(len(PHASES), np.float64)
    _check(lib().icd2s_get_phase_ms(st, _np(ms)))
    return dict(zip(PHASES, ms.tolist()))


def icd2s_kernel_launches() -> int:
    c = C.c_uint64()
    _check(lib().icd2s_kernel_launches(C.byref(c)))
    return int(c.value)


def icd2s_apply_flips_static(Q_dev: int, n: int, ld: int, replicas: int, flips_dev: int, x_dev: int, g_dev: int,
                             E_dev: int, stream=0) -> None:
    """Allocation-free flip write-back on caller-owned device buffers (see
    include/icd2s.h): for callers that cannot call cudaMalloc."""
    _check(lib().icd2s_apply_flips_static(C.c_void_p(Q_dev), n, ld, replicas, C.c_void_p(flips_dev),
                                          C.c_void_p(x_dev), C.c_void_p(g_dev), C.c_void_p(E_dev), _s(stream)))


class Tuning(C.Structure):
    _fields_ = [("tabu_variant", C.c_int32), ("anneal_warps_per_cta", C.c_int32), ("refresh_bn", C.c_int32),
                ("refresh_splits", C.c_int32), ("tabu_wide_keys", C.c_int32),
                ("tabu_rows", C.c_int32), ("anneal_scheme", C.c_int32), ("refresh_kind", C.c_int32),
                ("tabu_cluster", C.c_int32)]


def _tuning_dict(t):
    return dict(tabu_variant=t.tabu_variant, anneal_warps_per_cta=t.anneal_warps_per_cta,
                refresh_bn=t.refresh_bn, refresh_splits=t.refresh_splits, tabu_wide_keys=t.tabu_wide_keys,
                tabu_rows=t.tabu_rows, anneal_scheme=t.anneal_scheme, refresh_kind=t.refresh_kind,
                tabu_cluster=t.tabu_cluster)


def icd2s_set_tuning(st, tabu_variant: int = -1, anneal_warps_per_cta: int = 0, refresh_bn: int = 0,
                     refresh_splits: int = 0, tabu_wide_keys: int = 0, tabu_rows: int = 0,
                     anneal_scheme: int = 0, refresh_kind: int = 0, tabu_cluster: int = 0) -> None:
    t = Tuning(tabu_variant=tabu_variant, anneal_warps_per_cta=anneal_warps_per_cta, refresh_bn=refresh_bn,
               refresh_splits=refresh_splits, tabu_wide_keys=tabu_wide_keys, tabu_rows=tabu_rows,
               anneal_scheme=anneal_scheme, refresh_kind=refresh_kind, tabu_cluster=tabu_cluster)
    _check(lib().icd2s_set_tuning(st, C.byref(t)))


def icd2s_get_tuning(st) -> dict:
    t = Tuning()
    _check(lib().icd2s_get_tuning(st, C.byref(t)))
    return _tuning_dict(t)


def icd2s_refresh(st, rebuild: bool = False, stream=0) -> int:
    """Tensor-core recompute of all gains/energies; returns the number of
    entries that differ from the tracked ones (synchronises)."""
    bad = C.c_int32(0)
    _check(lib().icd2s_refresh(st, 1 if rebuild else 0, C.byref(bad), _s(stream)))
    return int(bad.value)


def icd2s_get_refresh_ms(st) -> float:
    ms = C.c_double(0.0)
    _check(lib().icd2s_get_refresh_ms(st, C.byref(ms)))
    return float(ms.value)


def icd2s_get_apply_ms(st) -> float:
    ms = C.c_double(0.0)
    _check(lib().icd2s_get_apply_ms(st, C.byref(ms)))
    return float(ms.value)


def icd2s_autotune(st, p: Params, stream=0) -> dict:
    t = Tuning()
    _check(lib().icd2s_autotune(st, C.byref(p), C.byref(t), _s(stream)))
    return _tuning_dict(t)


def icd2s_debug_refresh_stall(st, launches: int, wait_us: int) -> None:
    """Fault injection: the next `launches` refreshes skip their operand loads
    and time out after wait_us (see include/icd2s.h)."""
    _check(lib().icd2s_debug_refresh_stall(st, launches, wait_us))


def icd2s_mlp_set_tensor_cores(m, enable: bool = True) -> None:
    """The network's gradient on the tensor cores (BF16 operands, FP32 accumulation) or in FP32."""
    _check(lib().icd2s_mlp_set_tensor_cores(m, 1 if enable else 0))
