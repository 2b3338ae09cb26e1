#!/usr/bin/env python
"""Benchmark of the IC-D2S hot path on GB300.

A step is one whole outer iteration of Algorithm 2 on the device (Tabu
search, control parameters, subQUBO selection, the emulated Ising machine,
write-back, mutation, best update) over one synthetic solution set.  The
metric is spin-flip attempts of the emulated Ising machine per second of
step time (sweeps x subQUBO size x subQUBOs per step / step time).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference] [--workload NAME]
  python bench.py --ttt [--ttt-seeds S] [--ttt-budget ITERS] [--ttt-instances a,b]

The line also carries a time-to-target block (`ttt`, the metric's second
half): learned / batched selection against the plain method on the n = 5000,
50 % density instance, device-timed, 10 seeds.
The default workload is the Beasley-shaped instance (n = 2500, 10 % density,
int8 entries in [-100, 100]) with 128 replicas, subQUBOs of 64, 1024 sweeps,
alpha = 5n, c = 16 and a 1 % mutation rate.  Inputs are resident in HBM when
the timed region starts; L2 is flushed (a 256 MiB write, then a 256 MiB
read) before every timed step, outside the step's events.  `--impl reference` times the CPU oracle
(single thread, as it stands) on a bounded sample of the same workload.
Under torchrun the ranks solve one problem together: every rank holds 128
replicas of a set of 128 x N (a replica shard; weak scaling), and each outer
iteration adds the shards' column counts for gamma (one allreduce of n int32,
Eq. 8), the only exchange the method has on its data path.  Rank 0 prints
one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2502_13947_gb300.instances import make_qubo, random_solutions  # noqa: E402

WORKLOADS = {
    "beasley-like-n2500-d0.1-m64-z128": dict(
        n=2500, density=0.1, qseed=1, z=128, K=1, m_min=64, m_max=64, m_init=64, sweeps=1024, alpha=12500, c=16,
        T_max=1500.0, T_min=1.0, mut_mode=1, mut_rate=0.01),
}
DEFAULT_WORKLOAD = "beasley-like-n2500-d0.1-m64-z128"
METRIC = "spin-flip attempts/s"
UNIT = "attempts/s"
L2_FLUSH_BYTES = 256 << 20


class L2Flush:
    """Flushes the L2 between timed iterations: writes a buffer larger than L2,
    then reads another one, so the timed work starts with clean lines (the
    write alone would leave ~L2-size dirty lines whose write-back the next
    kernel would pay for)."""

    def __init__(self, torch):
        self.w = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
        self.r = torch.zeros(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")

    def __call__(self):
        self.w.zero_()
        self.r.max()


def attempts_per_step(w):
    # subQUBO sizes are drawn per (replica, group); the mean is exact for m_min == m_max
    return w["z"] * w["K"] * w["sweeps"] * (w["m_min"] + w["m_max"]) // 2


def max_over_ranks(dist, torch, seconds_or_ms, device):
    """The slowest rank's time (every rank gets it)."""
    tt = torch.tensor([float(seconds_or_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def whole_job_rate(world, units_per_rank_step, steps, seconds):
    """Units processed by all ranks (each holds the same number of replicas:
    weak scaling) per second of the slowest rank's time."""
    return world * units_per_rank_step * steps / seconds


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


def ncu_traffic(kernel_file, kernel, field="dram_bytes_per_launch"):
    """A per-launch counter (DRAM bytes by default) from the committed ncu
    summary, if the kernel's source is unchanged since the capture (else None)."""
    try:
        with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as f:
            tab = json.load(f)
        ent = tab.get(kernel)
        if not ent:
            return None
        src = os.path.join(ROOT, "paper_2502_13947_gb300", "csrc", kernel_file)
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()
        return ent.get(field) if ent.get("source_sha256") == h else None
    except (OSError, KeyError, ValueError):
        return None


# ----------------------------------------------------------------------------- clocks
CLOCK_Q = ("uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
           "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
           "clocks_event_reasons.sw_power_cap")


def start_clocks():
    try:
        return subprocess.Popen(["nvidia-smi", "--query-gpu=" + CLOCK_Q, "--format=csv,noheader,nounits", "-lms", "100"],
                                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
    except OSError:
        return None


def stop_clocks(proc, uuid):
    if proc is None:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
    proc.terminate()
    try:
        out, _ = proc.communicate(timeout=5)
    except subprocess.TimeoutExpired:
        proc.kill()
        out, _ = proc.communicate()
    sm, smax, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in out.splitlines():
        f = [x.strip() for x in line.split(",")]
        if len(f) < 9 or (uuid and f[0] != uuid):
            continue
        try:
            sm.append(float(f[1]))
            smax.append(float(f[2]))
        except ValueError:
            continue
        for nm, v in zip(names, f[5:9]):
            if v.lower().startswith("active"):
                reasons.add(nm)
    return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
            "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- oracle arm
def oracle_sample(w, z_sample, seed=9):
    """One oracle step on z_sample replicas of the workload; returns (seconds, attempts)."""
    from oracle import oracle as O
    O.build()
    Q = make_qubo(w["n"], w["density"], w["qseed"])
    prm = O.Params(z=z_sample, K=w["K"], m_min=w["m_min"], m_max=w["m_max"], m_init=w["m_init"], alpha=w["alpha"],
                   c=w["c"], sweeps=w["sweeps"], T_max=w["T_max"], T_min=w["T_min"], w1=65536, w2=65536, w3=32768,
                   mut_mode=w["mut_mode"], mut_rate=w["mut_rate"], patience=0, max_iters=1)
    S0 = random_solutions(w["n"], z_sample, 42)
    t0 = time.perf_counter()
    O.step(Q, prm, seed, 0, S0)
    dt = time.perf_counter() - t0
    return dt, z_sample * w["K"] * w["sweeps"] * (w["m_min"] + w["m_max"]) // 2


def n_core_ideal(single_core_rate):
    """The single-core oracle rate times the host's cores: an upper bound for a
    parallel CPU run, since the replicas of a phase are independent."""
    cores = os.cpu_count() or 1
    return {"n_core_ideal": {"value": single_core_rate * cores, "cores": cores,
                             "note": "upper bound: cores x the single-core rate (replicas are independent)"}}


def run_reference(args, w):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    per_replica = 0.15  # seconds of oracle time per replica-step on one core (measured order of magnitude)
    z_s = int(max(1, min(w["z"], 120.0 / max(1, args.steps + args.warmup) / per_replica)))
    for _ in range(args.warmup):
        oracle_sample(w, z_s)
    times, att = [], 0
    for _ in range(args.steps):
        dt, att = oracle_sample(w, z_s)
        times.append(dt)
    tot = sum(times)
    value = att * len(times) / tot
    sample = "one outer iteration of the workload on %d of its %d replicas per step (single-threaded C oracle)" % (
        z_s, w["z"])
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * tot / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": dict(workload=args.workload, **{k: w[k] for k in ("n", "density", "z", "K", "m_min", "m_max",
                                                                          "sweeps", "alpha", "c", "mut_rate")},
                           replicas_per_sample_step=z_s, l2="n/a (CPU)",
                           differs_from_gpu_line="only in the replicas sampled per step (%d of %d); every replica "
                                                 "of a phase does the same work, so attempts/s is comparable"
                                                 % (z_s, w["z"])),
            "cpu_baseline": dict({"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
                                 **n_core_ideal(value)),
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- dense refresh
REFRESH_WORKLOAD = dict(name="palubeckis-like-n7000-d1.0-R256", n=7000, density=1.0, qseed=7, z=256)


def measure_refresh(I, torch, peaks, stream, flush, reps=10):
    """The exact tensor-core refresh H = Q X^T on the dense n = 7000 instance
    with 256 replicas: kernel time (CUDA events on the launching stream, L2
    flushed before each call) against the measured BF16 peak."""
    w = REFRESH_WORKLOAD
    n, R = w["n"], w["z"]
    Q = make_qubo(n, w["density"], w["qseed"])
    q = I.icd2s_qubo_create(Q)
    st = I.icd2s_state_create(q, R, 11)
    sp = stream.cuda_stream
    try:
        I.icd2s_set_timing(st, True)
        bad = I.icd2s_refresh(st, False, sp)          # warm-up (builds the BF16 copies)
        mma, whole = [], []
        for _ in range(reps):
            with torch.cuda.stream(stream):
                flush()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
            bad += I.icd2s_refresh(st, False, sp)
            with torch.cuda.stream(stream):
                e1.record(stream)
            e1.synchronize()
            whole.append(e0.elapsed_time(e1))
            mma.append(I.icd2s_get_refresh_ms(st))
    finally:
        I.icd2s_state_destroy(st)
        I.icd2s_qubo_destroy(q)
    ms = sum(mma) / len(mma)
    flops = 2.0 * n * n * R
    tf = flops / (ms / 1000.0) / 1e12
    ld = (n + 127) // 128 * 128
    return {"kernel": "k_refresh_mma", "workload": w["name"], "bound": "tensor", "achieved": tf,
            "peak": peaks["bf16_tflops"], "unit": "TFLOP/s", "frac": tf / peaks["bf16_tflops"],
            "traffic": ncu_traffic("kernels_refresh.cu", "k_refresh_mma"),
            "algorithmic_flops_per_launch": flops, "algorithmic_bytes_per_launch": 2 * n * ld + 2 * R * ld + 4 * R * ld,
            "launch_ms": ms, "refresh_call_ms": sum(whole) / len(whole), "mismatches": bad,
            "peak_source": "MEASURED_PEAKS.json bf16_tflops (burst: the kernel is timed alone)"}


# The dense-refresh workload as a whole: Ising-machine rounds (selection, one
# batched anneal launch of R x K uneven subQUBOs, exact write-back) on the dense
# n = 7000 instance with 256 replicas, and every 64 rounds a tensor-core refresh
# of all gains and energies that checks the tracked values.
C4_WORKLOAD = dict(name="dense-n7000-d1.0-R256-K16-m32..256-refresh-every-64-rounds", n=7000, density=1.0, qseed=7,
                   z=256, K=16, m_min=32, m_max=256, sweeps=256, rounds=64)


def measure_c4(I, torch, stream):
    """Device time of 64 Ising-machine rounds and of the refresh that follows
    them (CUDA events on the launching stream), the refresh's share, and the
    anneal's attempt rate over the rounds."""
    w = C4_WORKLOAD
    n, R = w["n"], w["z"]
    q = I.icd2s_qubo_create(make_qubo(n, w["density"], w["qseed"]))
    st = I.icd2s_state_create(q, R, 5)
    p = I.icd2s_default_params(n, z=R, K=w["K"], m_min=w["m_min"], m_max=w["m_max"], m_init=64, sweeps=w["sweeps"])
    sp = stream.cuda_stream
    try:
        with torch.cuda.stream(stream):
            I.icd2s_tabu(st, n, p.c, sp)              # toggle counts for Delta (Eq. 7)
            I.icd2s_im_round(st, p, 0, sp)             # warm-up (tables, buffers)
            bad = I.icd2s_refresh(st, False, sp)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            ev[0].record(stream)
            for r in range(w["rounds"]):
                I.icd2s_im_round(st, p, 1 + r, sp)
            ev[1].record(stream)
        bad += I.icd2s_refresh(st, False, sp)         # the drift check (synchronises)
        with torch.cuda.stream(stream):
            ev[2].record(stream)
        ev[2].synchronize()
    finally:
        I.icd2s_state_destroy(st)
        I.icd2s_qubo_destroy(q)
    rounds_ms, refresh_ms = ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])
    attempts = w["rounds"] * R * w["K"] * w["sweeps"] * (w["m_min"] + w["m_max"]) / 2.0   # mean size
    return {"workload": w["name"], "rounds": w["rounds"], "rounds_ms": rounds_ms, "round_ms": rounds_ms / w["rounds"],
            "refresh_call_ms": refresh_ms, "refresh_share": refresh_ms / (rounds_ms + refresh_ms),
            "anneal_attempts_per_s_expected_sizes": attempts / (rounds_ms / 1000.0), "mismatches": bad,
            "note": "a round = selection + one batched anneal launch + write-back; the refresh checks all "
                    "256 x 7000 gains and 256 energies (0 mismatches expected)"}


# The proposal network at the learned-selection workload's size: scores of
# every variable of 32 replicas of n = 10 000 (320 000 rows), and training
# steps on 8192-row batches, with the gradient on the CUDA cores (FP32) and on
# the tensor cores (BF16 operands, FP32 accumulation).
MLP_WORKLOAD = dict(name="learned-n10000-z32", rows=320000, batch=8192, steps=50)


def measure_mlp(I, torch, stream, reps=10):
    w = MLP_WORKLOAD
    g = torch.Generator(device="cpu").manual_seed(3)
    F = torch.rand((w["rows"], 6), generator=g).cuda()
    y = (torch.rand(w["rows"], generator=g) < 0.1).to(torch.uint8).cuda()
    out = torch.empty(w["rows"], dtype=torch.float32, device="cuda")
    m = I.icd2s_mlp_create(1)
    sp = stream.cuda_stream
    res = {"workload": w["name"], "score_rows": w["rows"], "train_batch": w["batch"]}
    try:
        def timed(fn):
            with torch.cuda.stream(stream):
                fn()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(reps):
                    fn()
                e1.record(stream)
            e1.synchronize()
            return e0.elapsed_time(e1) / reps
        res["score_ms"] = timed(lambda: I.icd2s_mlp_score(m, F.data_ptr(), w["rows"], out.data_ptr(), sp))
        for tc in (False, True):
            I.icd2s_mlp_set_tensor_cores(m, tc)
            ms = timed(lambda: I.icd2s_mlp_train(m, F.data_ptr(), y.data_ptr(), w["rows"], steps=w["steps"],
                                                 batch=w["batch"], lr=1e-3, stream=sp))
            res["train_step_ms_" + ("tensor_cores" if tc else "fp32")] = ms / w["steps"]
    finally:
        I.icd2s_mlp_destroy(m)
    flops = 2 * 8960
    res["score_gflops"] = flops * w["rows"] / (res["score_ms"] / 1000) / 1e9
    return res


APPLY_WORKLOAD = dict(name="gain-update-n16384-R16-disjoint1024", n=16384, density=1.0, qseed=5, R=16)


def measure_apply(I, torch, peaks, stream, flush, reps=10):
    """The exact gain write-back (icd2s_apply_flips_update_gains) streaming
    every row of Q once: n = 16 384, 16 replicas, replica p flips the 1024
    variables i = p (mod 16), so the flip sets are disjoint and no row is
    reused (Q is 268 MB, twice the L2).  The kernel time comes from CUDA
    events the library records around the write-back kernel on the launching
    stream; call_ms adds the mask compaction (events around the call); L2 is
    flushed before each call."""
    w = APPLY_WORKLOAD
    n, R = w["n"], w["R"]
    Q = make_qubo(n, w["density"], w["qseed"])
    q = I.icd2s_qubo_create(Q)
    del Q
    st = I.icd2s_state_create(q, R, 3)
    sp = stream.cuda_stream
    mask = np.zeros((R, n), np.uint8)
    for p in range(R):
        mask[p, p::R] = 1
    mask_d = torch.from_numpy(mask).cuda()
    ms, kms = [], []
    try:
        I.icd2s_set_timing(st, True)
        with torch.cuda.stream(stream):
            I.icd2s_apply_flips_update_gains(st, mask_d.data_ptr(), sp)   # warm-up
        for _ in range(reps):
            with torch.cuda.stream(stream):
                flush()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                I.icd2s_apply_flips_update_gains(st, mask_d.data_ptr(), sp)
                e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
            kms.append(I.icd2s_get_apply_ms(st))
    finally:
        I.icd2s_state_destroy(st)
        I.icd2s_qubo_destroy(q)
    ld = (n + 127) // 128 * 128
    flips = int(mask.sum())
    # per (replica, flip): the flipped row of Q (ld bytes streamed); per
    # replica: the mask row, g read + written, x read + written
    nbytes = flips * ld + R * (n + 8 * ld + 2 * ld)
    t = sum(kms) / len(kms)
    tc = sum(ms) / len(ms)
    gbs = nbytes / (t / 1000.0) / 1e9
    return {"kernel": "k_apply", "workload": w["name"], "bound": "hbm", "achieved": gbs, "peak": peaks["hbm_gbs"],
            "unit": "GB/s", "frac": gbs / peaks["hbm_gbs"], "traffic": ncu_traffic("kernels_update.cu", "k_apply"),
            "algorithmic_bytes_per_launch": nbytes, "launch_ms": t, "call_ms": tc,
            "call_frac": nbytes / (tc / 1000.0) / 1e9 / peaks["hbm_gbs"],
            "peak_source": "MEASURED_PEAKS.json hbm_gbs (burst: the call is timed alone)"}


TABU_WORKLOAD = dict(name="tabu-n5000-d0.5-z32-alpha5n", n=5000, density=0.5, qseed=1, z=32, alpha_per_n=5,
                     c_div=150)


def measure_tabu(I, torch, peaks, stream, flush, reps=3):
    """One Tabu search (Algorithm 1) of every replica at the time-to-target
    shape: n = 5000, rho = 0.5 (gain bound too wide for the compact keys on
    indices: the keys on parity labels), 32 replicas, alpha = 5n.  Library
    events around the call on the launching stream, L2 flushed before each."""
    w = TABU_WORKLOAD
    n, z = w["n"], w["z"]
    alpha, c = w["alpha_per_n"] * n, max(2, n // w["c_div"])
    Q = make_qubo(n, w["density"], w["qseed"])
    q = I.icd2s_qubo_create(Q)
    bound = I.icd2s_qubo_gain_bound(q)
    st = I.icd2s_state_create(q, z, 5)
    X0 = random_solutions(n, z, 3)
    sp = stream.cuda_stream
    ms = []
    try:
        for r in range(reps + 1):
            with torch.cuda.stream(stream):
                I.icd2s_state_load(st, X0, stream=sp)
                flush()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                I.icd2s_tabu(st, alpha, c, sp)
                e1.record(stream)
            e1.synchronize()
            if r > 0:   # the first call is the warm-up
                ms.append(e0.elapsed_time(e1))
    finally:
        I.icd2s_state_destroy(st)
        I.icd2s_qubo_destroy(q)
    t = sum(ms) / len(ms)
    return {"kernel": "k_tabu", "workload": w["name"], "gain_bound": bound, "alpha": alpha, "c": c, "launch_ms": t,
            "moves_per_s": z * alpha / (t / 1000.0), "us_per_move": t * 1000.0 / alpha}


# ----------------------------------------------------------------------------- GPU arm
def run_only(args):
    """One measurement alone (for profiling commands): --only apply|refresh|tabu."""
    import torch

    from paper_2502_13947_gb300 import build as B
    from paper_2502_13947_gb300 import icd2s as I
    torch.cuda.set_device(0)
    if not B.up_to_date():
        B.build()
    peaks, _ = measured_peaks()
    stream = torch.cuda.Stream()
    flush = L2Flush(torch)
    fn = {"apply": measure_apply, "refresh": measure_refresh, "tabu": measure_tabu}[args.only]
    print(json.dumps(fn(I, torch, peaks, stream, flush, reps=args.steps)), flush=True)


def run_gpu(args, w):
    import torch
    import torch.distributed as dist

    from paper_2502_13947_gb300 import build as B
    from paper_2502_13947_gb300 import icd2s as I

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    if not B.up_to_date():
        if rank == 0:
            B.build()
        if world > 1:
            dist.barrier()
    dev_uuid = None
    try:
        dev_uuid = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        pass

    n, z = w["n"], w["z"]              # z replicas per GPU
    z_total = z * world
    Q = make_qubo(n, w["density"], w["qseed"])   # one problem; its replica set is sharded over the ranks
    p = I.icd2s_default_params(n, z=z_total, K=w["K"], m_min=w["m_min"], m_max=w["m_max"], m_init=w["m_init"],
                               sweeps=w["sweeps"], alpha=w["alpha"], c=w["c"], T_max=w["T_max"], T_min=w["T_min"],
                               mut_mode=w["mut_mode"], mut_rate=w["mut_rate"], patience=0, max_iters=1 << 30)
    q = I.icd2s_qubo_create(Q)
    stream = torch.cuda.Stream()
    sp = stream.cuda_stream
    flush = L2Flush(torch)
    sharded = None
    if world > 1:
        from paper_2502_13947_gb300.shard import ShardedState
        sharded = ShardedState(I, torch, dist, q, n, z_total, 7)
        st = sharded.st
    else:
        st = I.icd2s_state_create(q, z, 7)

    def step(t):  # enqueued on `stream` (the current stream inside the caller's context)
        if sharded:
            sharded.step(p, t)
        else:
            I.icd2s_step(st, p, t, sp)

    with torch.cuda.stream(stream):
        if sharded:
            sharded.initial_pass(p)
        else:
            I.icd2s_initial_pass(st, p, sp)
            I.icd2s_best_update(st, sp)
    torch.cuda.synchronize()
    I.icd2s_set_timing(st, True)
    t = 0
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step(t)
            t += 1
    torch.cuda.synchronize()

    phase_tot = dict.fromkeys(I.PHASES, 0.0)
    step_ms = []
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = start_clocks() if rank == 0 else None
    time.sleep(0.25 if clocks else 0)
    launches0 = I.icd2s_kernel_launches()
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush()                             # L2 flush, outside the step's events
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step(t)
            e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        for k, v in I.icd2s_get_phase_ms(st).items():
            phase_tot[k] += v
        t += 1
    launches = I.icd2s_kernel_launches() - launches0
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = stop_clocks(clocks, dev_uuid) if rank == 0 else None
    total_ms = sum(step_ms)
    if world > 1:
        total_ms = max_over_ranks(dist, torch, total_ms, "cuda")
    att = attempts_per_step(w)
    value = whole_job_rate(world, att, args.steps, total_ms / 1000.0)

    # end to end through the host-buffer entry point (pinned host memory, copies inside the timed region)
    e2e_steps = max(1, min(args.steps, 10))
    x_in = torch.empty((z, n), dtype=torch.uint8, pin_memory=True).numpy()
    x_out = torch.empty((z, n), dtype=torch.uint8, pin_memory=True).numpy()
    E_out = torch.empty(z, dtype=torch.int64, pin_memory=True).numpy()
    x_in[:] = random_solutions(n, z, 5 + rank)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    e2e_s = 0.0
    for _ in range(e2e_steps):
        t0 = time.perf_counter()
        if sharded:   # the same copies around the shard's step: x in, then x and E out
            with torch.cuda.stream(stream):
                I.icd2s_state_load(st, x_in, stream=sp)
                step(t)
            I.icd2s_get_state(st, z, n, x=x_out, E=E_out, want_g=False)
        else:
            I.icd2s_step_host(st, p, t, x_in, x_out, E_out, sp)
        e2e_s += time.perf_counter() - t0
        x_in[:] = x_out
        t += 1
    if world > 1:
        e2e_s = max_over_ranks(dist, torch, e2e_s, "cuda")
    e2e_value = whole_job_rate(world, att, e2e_steps, e2e_s)

    if sharded:
        sharded.close()
    else:
        I.icd2s_state_destroy(st)
    I.icd2s_qubo_destroy(q)
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    peaks, peak_src = measured_peaks()
    refresh = None if args.no_refresh else measure_refresh(I, torch, peaks, stream, flush)
    apply_rf = None if args.no_refresh else measure_apply(I, torch, peaks, stream, flush)
    c4 = None if args.no_refresh else measure_c4(I, torch, stream)
    mlp = None if args.no_refresh else measure_mlp(I, torch, stream)
    K = args.steps
    phase_avg = {k: v / K for k, v in phase_tot.items()}
    ld = (n + 127) // 128 * 128
    # Tabu (Algorithm 1): one row of Q (n bytes) per iteration per replica, plus
    # the replica state read and written once (g, C, T int32; x bytes)
    tabu_bytes = z * w["alpha"] * n + z * ld * (4 + 4 + 4 + 4 + 1 + 1)
    tabu_s = phase_avg["tabu"] / 1000.0
    tabu_gbs = tabu_bytes / tabu_s / 1e9
    roofline = {"kernel": "k_tabu", "bound": "hbm", "achieved": tabu_gbs, "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "frac": tabu_gbs / peaks["hbm_gbs"],
                "traffic": ncu_traffic("kernels_tabu.cu", "k_tabu"),
                "algorithmic_bytes_per_launch": tabu_bytes, "launch_ms": phase_avg["tabu"],
                "peak_source": peak_src + " (MEASURED_PEAKS.json hbm_gbs)" if peak_src == "measured" else peak_src}
    # The Tabu kernel's own limit: one CTA per replica runs a dependent chain per
    # move, and its SMs issue at a fraction of one warp instruction per cycle per
    # sub-partition (warp instructions per launch from the ncu capture of one
    # launch, profiles/; the same peak rule as the anneal's below).
    sms_t = torch.cuda.get_device_properties(local).multi_processor_count
    mhz_t = (clk or {}).get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    inst_t = ncu_traffic("kernels_tabu.cu", "k_tabu", "warp_instructions_per_launch")
    used_t = min(z, sms_t)
    roofline["issue"] = {
        "warp_instructions_per_launch": inst_t,
        "achieved": (inst_t / tabu_s / 1e9) if inst_t else None,
        "peak": sms_t * 4 * mhz_t / 1000.0, "unit": "G warp-instructions/s",
        "frac": (inst_t / tabu_s / 1e9) / (sms_t * 4 * mhz_t / 1000.0) if inst_t else None,
        "frac_of_sms_used": (inst_t / tabu_s / 1e9) / (used_t * 4 * mhz_t / 1000.0) if inst_t else None,
        "sms_used": used_t,
        "cycles_per_move": tabu_s * mhz_t * 1e6 / w["alpha"],
    }
    anneal_rate = att / (phase_avg["anneal"] / 1000.0)
    # The Ising machine's anneal (a7): a sequential Metropolis chain per subQUBO,
    # bound by integer issue.  Warp instructions per attempt come from the ncu
    # capture of one launch (profiles/); the peak is every SM sub-partition
    # issuing one warp instruction per cycle at the sampled SM clock.
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    mhz = (clk or {}).get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    inst = ncu_traffic("kernels_anneal.cu", "k_anneal", "warp_instructions_per_launch")
    positions_per_warp = w["sweeps"] * w["m_max"]   # one warp per subQUBO of m_max positions (m_min == m_max)
    roofline_anneal = {
        "kernel": "k_anneal", "bound": "alu", "unit": "G warp-instructions/s",
        "peak": sms * 4 * mhz / 1000.0,
        "peak_rule": "%d SMs x 4 sub-partitions x 1 warp instruction per cycle x %.0f MHz (sampled SM clock)" % (
            sms, mhz),
        "attempts_per_s": anneal_rate,
        "cycles_per_position": phase_avg["anneal"] / 1000.0 * mhz * 1e6 / positions_per_warp,
        "warp_instructions_per_attempt": (inst / att) if inst else None,
        "achieved": (inst / att * anneal_rate / 1e9) if inst else None,
        "warps": z * w["K"],
        "note": "one warp per subQUBO: %d warps can use at most %d of the %d sub-partitions" % (
            z * w["K"], min(z * w["K"], sms * 4), sms * 4),
    }
    roofline_anneal["frac"] = (roofline_anneal["achieved"] / roofline_anneal["peak"]
                               if roofline_anneal["achieved"] else None)

    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        dt, a = oracle_sample(w, z)
        cpu = {"value": a / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": "one whole outer iteration of the workload (all %d replicas), single-threaded C oracle, "
                         "%.1f s" % (z, dt)}
        cpu.update(n_core_ideal(a / dt))
    ttt = None if (args.no_ttt or world > 1) else ttt_block(I, torch)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": args.warmup,
        "ms_per_step": total_ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int32", "data": "synthetic",
        "config": {"workload": args.workload, "n": n, "density": w["density"], "z": z_total, "z_per_gpu": z,
                   "K": w["K"],
                   "m_min": w["m_min"], "m_max": w["m_max"], "sweeps": w["sweeps"], "alpha": w["alpha"],
                   "c": w["c"], "mutation_rate": w["mut_rate"], "T_max": w["T_max"], "T_min": w["T_min"],
                   "attempts_per_step": att,
                   "parallelism": ("replica shards of one problem, %d per GPU; one allreduce of n int32 column "
                                   "counts per iteration (gamma, Eq. 8)" % z) if world > 1 else "1 GPU",
                   "l2": "flushed before every timed step (256 MiB write + 256 MiB read, outside the step events)"},
        "roofline": roofline,
        "roofline_refresh": refresh,
        "roofline_apply": apply_rf,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": z * n, "d2h_bytes_per_step": z * n + 8 * z,
                "steps": e2e_steps, "api": "icd2s_step_host"},
        "gpu_launches": launches,
        "clocks": clk,
        "phase_ms": phase_avg,
        "anneal_kernel_attempts_per_s": anneal_rate,
        "roofline_anneal": roofline_anneal,
        "c4": c4,
        "mlp": mlp,
        "ttt": ttt,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


# ----------------------------------------------------------------------------- time to target
# Second metric: device-timed time to a target energy, learned / batched
# selection against the plain method, on one GPU.  Instances are the
# generator's dense-ish synthetic stand-ins (n = 5000 and 10 000, 50 %
# density); the target E* of an instance is the best energy of three plain
# runs ten times as long as the measured ones (run seeds 100-102); every
# method then runs from seeds 0..S-1 until its best energy is <= E* or the
# iteration budget is spent (a miss, censored at the budget).
TTT_INSTANCES = {"n5000-d0.5": dict(n=5000, density=0.5, qseed=0),
                 "n10000-d0.5": dict(n=10000, density=0.5, qseed=0)}
TTT_METHODS = {  # (K, m_min, m_max, select_mode, ablation, im_order, alpha / n)
    "plain": (1, 64, 64, 0, 0, 0, 5),
    "batched": (16, 32, 256, 0, 0, 0, 5),
    "learned": (1, 64, 64, 1, 0, 0, 5),
    "learned+batched": (16, 32, 256, 1, 0, 0, 5),
    "hybrid+batched": (16, 32, 256, 2, 0, 0, 5),
    "batched K=4": (4, 32, 256, 0, 0, 0, 5),           # fewer subQUBOs per solution: a larger mutation
    "learned+batched K=4": (4, 32, 256, 1, 0, 0, 5),
    "batched GS": (16, 32, 256, 0, 0, 1, 5),          # Gauss-Seidel order of the 16 subQUBOs
    "learned+batched GS": (16, 32, 256, 1, 0, 1, 5),
    "No_IM": (1, 64, 64, 0, 1, 0, 5),      # the simplified versions of Section 4
    "No_SM": (1, 64, 64, 0, 2, 0, 5),
    "Tabu-only a=20n": (1, 64, 64, 0, 1, 0, 20),  # classical comparator: Tabu + mutation at the
                                                  # alpha = 20n the paper gives the Tabu-only solver
}
# improvement logs of the plain method for training: shapes of the n = 64
# dense, n = 2500 sparse and n = 5000 batched workloads, and the plain method in
# the time-to-target block's regime (n = 5000, alpha = n); instance seeds 200+,
# never the measured instance.  Fields: n, density, z, K, m_min, m_max,
# iterations, alpha / n.
TTT_LOG_SHAPES = ((64, 1.0, 8, 1, 16, 16, 200, 5), (2500, 0.1, 128, 1, 64, 64, 40, 5),
                  (5000, 0.5, 32, 16, 32, 256, 40, 5), (5000, 0.5, 32, 1, 64, 64, 40, 1))


def ttt_params(I, n, K, m_min, m_max, mode, iters, z=32):
    p = I.icd2s_default_params(n)
    p.z, p.K, p.m_min, p.m_max, p.m_init = z, K, m_min, m_max, 64 if n >= 64 else n
    p.alpha, p.c, p.sweeps, p.T_max, p.T_min = 5 * n, max(2, n // 150), 256, 2000.0, 1.0
    p.mut_mode, p.patience, p.max_iters, p.select_mode, p.use_graph = 0, 0, iters, mode, 1
    return p


def ttt_train(I, torch, steps=3000, batch=8192, runs=4):
    """Collects improvement logs of plain runs and trains the network on the GPU."""
    Fs, ys, entries = [], [], 0
    for (n, rho, z, K, m_min, m_max, iters, amul) in TTT_LOG_SHAPES:
        for r in range(runs):
            q = I.icd2s_qubo_create(make_qubo(n, rho, 200 + r))
            p = ttt_params(I, n, K, m_min, m_max, 0, iters, z=z)
            p.m_init = min(m_max, 64)
            p.alpha = amul * n
            st = I.icd2s_state_create(q, z, 200 + r)
            I.icd2s_log_enable(st, 512)
            I.icd2s_state_run(st, n, p)
            e, cap = I.icd2s_log_info(st)
            cnt = min(e, cap)
            if cnt:
                F = torch.empty((cnt, n, 6), dtype=torch.float32, device="cuda")
                y = torch.empty((cnt, n), dtype=torch.uint8, device="cuda")
                I.icd2s_log_copy_device(st, F.data_ptr(), y.data_ptr())
                Fs.append(F.reshape(-1, 6))
                ys.append(y.reshape(-1))
                entries += cnt
            I.icd2s_state_destroy(st)
            I.icd2s_qubo_destroy(q)
    F = torch.cat(Fs).contiguous()
    y = torch.cat(ys).contiguous()
    pos = float(y.float().mean())
    pw = (1.0 - pos) / max(pos, 1e-9)
    m = I.icd2s_mlp_create(1)
    losses = I.icd2s_mlp_train(m, F.data_ptr(), y.data_ptr(), F.shape[0], steps=steps, batch=batch, lr=2e-3,
                               pos_weight=pw)
    info = dict(entries=entries, rows=int(F.shape[0]), positive_rate=round(pos, 5), pos_weight=round(pw, 3),
                steps=steps, batch=batch, loss_first=round(float(losses[:20].mean()), 4),
                loss_last=round(float(losses[-20:].mean()), 4))
    return m, info


def ttt_target(I, q, n, budget, alpha_mult=5):
    """E* of an instance: the best energy of three plain runs ten times as long as
    the measured ones (run seeds 100-102)."""
    longs = []
    for s in (100, 101, 102):
        p = ttt_params(I, n, 1, 64, 64, 0, 10 * budget)
        p.alpha = alpha_mult * n
        longs.append(I.icd2s_run(q, p, s)["best_E"])
    return min(longs), longs


def ttt_methods(I, q, n, mlp, E_star, methods, seeds, budget, alpha_mult=None):
    """Every method from run seeds 0..seeds-1 until best <= E* or the budget is
    spent: device time to the target (CUDA events, Call_IM_Solution_Set
    included), hits, iterations.  alpha_mult overrides each method's alpha / n."""
    res = {}
    for meth in methods:
        K, m_min, m_max, mode, ablation, order, amul = TTT_METHODS[meth]
        per = []
        for seed in range(seeds):
            p = ttt_params(I, n, K, m_min, m_max, mode, budget)
            p.ablation, p.im_order, p.alpha = ablation, order, (alpha_mult or amul) * n
            p.stop_at_target, p.target_E = 1, E_star
            st = I.icd2s_state_create(q, p.z, seed)
            if mode:
                I.icd2s_state_set_mlp(st, mlp)
            r = I.icd2s_state_run(st, n, p)
            I.icd2s_state_destroy(st)
            per.append(dict(seed=seed, hit_iter=r["hit_iter"], ttt_ms=round(r["ttt_ms"], 2), best_E=r["best_E"],
                            ms_per_iter=round(r["device_ms"] / max(r["iters"], 1), 2)))
        hits = [x["ttt_ms"] for x in per if x["hit_iter"] >= 0]
        cens = sorted(hits + [float("inf")] * (len(per) - len(hits)))
        med = cens[len(cens) // 2] if len(cens) % 2 else 0.5 * (cens[len(cens) // 2 - 1] + cens[len(cens) // 2])
        its = sorted(x["hit_iter"] + 1 if x["hit_iter"] >= 0 else budget + 1 for x in per)
        res[meth] = dict(median_ttt_ms=None if med == float("inf") else round(med, 2),
                         success=len(hits), runs=len(per), median_iterations=its[len(its) // 2],
                         mean_ms_per_iter=round(statistics.mean(x["ms_per_iter"] for x in per), 2),
                         per_seed=per)
    return res


# the time-to-target block of the default bench line: n = 5000, 50 % density,
# a Tabu search of alpha = n per iteration, so that the plain method needs
# several iterations to reach E* (with alpha = 5n every method reaches it in
# one to four)
TTT_DEFAULT = dict(instance="n5000-d0.5", methods=("plain", "learned", "batched", "learned+batched", "batched K=4",
                                                   "learned+batched K=4"), seeds=10, budget=30, alpha_mult=1)


def ttt_block(I, torch):
    """Time to target of learned / batched selection against the plain method
    (the default bench line's second metric)."""
    t0 = time.time()
    mlp, train_info = ttt_train(I, torch)
    spec = TTT_INSTANCES[TTT_DEFAULT["instance"]]
    n, am, budget = spec["n"], TTT_DEFAULT["alpha_mult"], TTT_DEFAULT["budget"]
    q = I.icd2s_qubo_create(make_qubo(n, spec["density"], spec["qseed"]))
    try:
        E_star, longs = ttt_target(I, q, n, budget, am)
        res = ttt_methods(I, q, n, mlp, E_star, TTT_DEFAULT["methods"], TTT_DEFAULT["seeds"], budget, am)
    finally:
        I.icd2s_qubo_destroy(q)
        I.icd2s_mlp_destroy(mlp)
    summary = {}
    for m, r in res.items():
        per = r.pop("per_seed")
        r["iterations"] = [x["hit_iter"] + 1 if x["hit_iter"] >= 0 else -1 for x in per]  # per seed, -1 = miss
        summary[m] = r
    def beats(a, b):   # more runs reach E*, or as many and a lower median device time
        return bool(a["success"] > b["success"] or
                    (a["success"] == b["success"] and a["median_ttt_ms"] is not None and
                     (b["median_ttt_ms"] is None or a["median_ttt_ms"] < b["median_ttt_ms"])))
    pl = summary["plain"]
    better = {"K=16": beats(summary["learned+batched"], pl), "K=4": beats(summary["learned+batched K=4"], pl)}
    network = {"K=1": beats(summary["learned"], pl), "K=16": beats(summary["learned+batched"], summary["batched"]),
               "K=4": beats(summary["learned+batched K=4"], summary["batched K=4"])}
    return {"metric": "time-to-target energy", "unit": "ms", "higher_is_better": False,
            "instance": TTT_DEFAULT["instance"], "target_E": E_star, "target_runs": longs,
            "target_rule": "best of 3 plain runs of 10x the budget (seeds 100-102)",
            "params": "z=32, alpha=%dn, c=n/150, 256 sweeps, T 2000->1, Eq. 5 mutation; learned / batched as in "
                      "--ttt" % am,
            "seeds": TTT_DEFAULT["seeds"], "budget_iters": budget, "methods": summary,
            "learned_batched_beats_plain": better, "learned_beats_same_batch_without_network": network,
            "train": train_info, "wall_s": round(time.time() - t0, 1)}


def run_ttt(args):
    import torch
    from paper_2502_13947_gb300 import icd2s as I
    if not torch.cuda.is_available():
        raise SystemExit("time-to-target needs a CUDA GPU")
    torch.cuda.set_device(0)
    t0 = time.time()
    mlp, train_info = ttt_train(I, torch)
    results = {}
    for name in args.ttt_instances.split(","):
        spec = TTT_INSTANCES[name]
        n = spec["n"]
        q = I.icd2s_qubo_create(make_qubo(n, spec["density"], spec["qseed"]))
        am = args.ttt_alpha
        E_star, longs = ttt_target(I, q, n, args.ttt_budget, am)
        res = dict(target_E=E_star, target_runs=longs, budget_iters=args.ttt_budget, alpha="%dn" % am)
        res.update(ttt_methods(I, q, n, mlp, E_star, list(TTT_METHODS), args.ttt_seeds, args.ttt_budget,
                               None if am == 5 else am))
        I.icd2s_qubo_destroy(q)
        results[name] = res
    I.icd2s_mlp_destroy(mlp)
    line = {"metric": "time-to-target energy", "unit": "ms", "higher_is_better": False, "n_gpus": 1,
            "data": "synthetic", "dtype": "int32/int64 (network: bf16 weights, f32)",
            "config": {"workload": "time-to-target, z=32, alpha=%dn, c=n/150, 256 sweeps, T 2000->1, Eq. 5 mutation"
                                   % args.ttt_alpha,
                       "methods": {k: dict(K=v[0], m_min=v[1], m_max=v[2], select_mode=v[3], ablation=v[4],
                                           im_order=v[5], alpha=f"{v[6]}n")
                                   for k, v in TTT_METHODS.items()}},
            "train": train_info, "results": results, "wall_s": round(time.time() - t0, 1)}
    print(json.dumps(line), flush=True)


SWEEP_PARAMS = {  # one parameter at a time around the plain method (z = 32, alpha = 5n, c = n/150)
    "z": (8, 16, 32, 64),
    "alpha/n": (1, 2, 5, 10),
    "c*150/n": (0.5, 1, 2, 5),
}


def run_sweep(args):
    """Time to target of the plain method as z, alpha and c vary (the
    parameter studies of Section 4 on a synthetic instance)."""
    import torch
    from paper_2502_13947_gb300 import icd2s as I
    if not torch.cuda.is_available():
        raise SystemExit("the parameter sweep needs a CUDA GPU")
    torch.cuda.set_device(0)
    t0 = time.time()
    spec = TTT_INSTANCES["n5000-d0.5"]
    n = spec["n"]
    q = I.icd2s_qubo_create(make_qubo(n, spec["density"], spec["qseed"]))
    longs = [I.icd2s_run(q, ttt_params(I, n, 1, 64, 64, 0, 10 * args.ttt_budget), s)["best_E"]
             for s in (100, 101, 102)]
    E_star = min(longs)
    results = {}
    for name, values in SWEEP_PARAMS.items():
        for v in values:
            per = []
            for seed in range(args.ttt_seeds):
                z = v if name == "z" else 32
                p = ttt_params(I, n, 1, 64, 64, 0, args.ttt_budget, z=z)
                if name == "alpha/n":
                    p.alpha = v * n
                if name == "c*150/n":
                    p.c = max(2, int(v * n / 150))
                p.stop_at_target, p.target_E = 1, E_star
                st = I.icd2s_state_create(q, p.z, seed)
                r = I.icd2s_state_run(st, n, p)
                I.icd2s_state_destroy(st)
                per.append((r["hit_iter"], r["ttt_ms"], r["device_ms"] / max(r["iters"], 1)))
            hits = sorted(t for h, t, _ in per if h >= 0)
            cens = hits + [float("inf")] * (len(per) - len(hits))
            med = cens[len(cens) // 2] if len(cens) % 2 else 0.5 * (cens[len(cens) // 2 - 1] + cens[len(cens) // 2])
            results["%s=%s" % (name, v)] = dict(success=len(hits), runs=len(per),
                                                median_ttt_ms=None if med == float("inf") else round(med, 2),
                                                iterations=[h + 1 if h >= 0 else -1 for h, _, _ in per],
                                                mean_ms_per_iter=round(statistics.mean(m for _, _, m in per), 2))
    I.icd2s_qubo_destroy(q)
    line = {"metric": "time-to-target energy, parameter sweep", "unit": "ms", "higher_is_better": False,
            "n_gpus": 1, "data": "synthetic",
            "config": {"workload": "n5000-d0.5 plain method (K=1, m=64, 256 sweeps, T 2000->1, Eq. 5 mutation)",
                       "defaults": "z=32, alpha=5n, c=n/150", "budget_iters": args.ttt_budget,
                       "target_E": E_star, "target_runs": longs},
            "results": results, "wall_s": round(time.time() - t0, 1)}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-refresh", action="store_true",
                    help="skip the tensor-core refresh and the write-back roofline measurements")
    ap.add_argument("--only", choices=["apply", "refresh", "tabu"], help="run one kernel measurement alone (profiling)")
    ap.add_argument("--ttt", action="store_true", help="time to target: learned / batched vs plain selection")
    ap.add_argument("--no-ttt", action="store_true", help="leave the time-to-target block out of the bench line")
    ap.add_argument("--ttt-seeds", type=int, default=10)
    ap.add_argument("--ttt-budget", type=int, default=30, help="outer iterations per measured run")
    ap.add_argument("--ttt-instances", default="n5000-d0.5,n10000-d0.5")
    ap.add_argument("--ttt-alpha", type=int, default=5, help="Tabu search length alpha / n of every method")
    ap.add_argument("--sweep", action="store_true", help="time to target as z, alpha and c vary (n = 5000)")
    args = ap.parse_args()
    w = WORKLOADS[args.workload]
    if args.only:
        run_only(args)
    elif args.ttt:
        run_ttt(args)
    elif args.sweep:
        run_sweep(args)
    elif args.impl == "reference":
        run_reference(args, w)
    else:
        run_gpu(args, w)


if __name__ == "__main__":
    main()
