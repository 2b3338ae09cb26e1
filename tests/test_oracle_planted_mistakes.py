"""The oracle's pins catch plausible mistakes.  Each case plants one mistake
in a copy of the oracle's C source -- a dropped term or factor, a wrong sign,
index, constant or comparison, an off-by-one -- builds it, and runs the
oracle's pin tests (test_oracle_core, test_oracle_method,
test_oracle_learned) against that build: at least one pin must fail.  The
unmodified copy, built the same way, passes them all, so a failure is the
planted mistake's and not the harness's.  The double-precision network
reference (oracle/mlp_ref.py) gets the same treatment against the
learned-selection pins, its mutated copy preloaded by a one-line pytest
plugin.  (The layout of the random streams is a convention both
implementations share, not arithmetic the paper fixes; GPU parity covers
it.)  CPU only."""
import concurrent.futures as cf
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "icd2s_oracle.c")
PINS = ["tests/test_oracle_core.py", "tests/test_oracle_method.py", "tests/test_oracle_learned.py"]

# (what the mistake is, text in the oracle, replacement)
MISTAKES = [
    ("Eq. 1 without the linear (diagonal) term",
     "        f += (int64_t)Q[(int64_t)i * n + i] * x[i];", "        f += 0 * x[i];"),
    ("Eq. 1 pair sum including i = j",
     "            if (j != i)\n                f += (int64_t)Q[(int64_t)i * n + j] * x[i] * x[j];",
     "            f += (int64_t)Q[(int64_t)i * n + j] * x[i] * x[j];"),
    ("gain without the symmetric factor 2 (reading S1)",
     "(Q[(int64_t)k * n + k] + 2 * s)", "(Q[(int64_t)k * n + k] + s)"),
    ("gain sign (1 - x) instead of (1 - 2x)",
     "g[k] = (int32_t)((1 - 2 * (int64_t)x[k])", "g[k] = (int32_t)((1 - (int64_t)x[k])"),
    ("Tabu update without the moved variable's sign (reading S2)",
     "dx[j] += 2 * Q[(int64_t)i * n + j] * si * (1 - 2 * x[j]);",
     "dx[j] += 2 * Q[(int64_t)i * n + j] * (1 - 2 * x[j]);"),
    ("Tabu update without the factor 2",
     "dx[j] += 2 * Q[(int64_t)i * n + j] * si * (1 - 2 * x[j]);",
     "dx[j] += Q[(int64_t)i * n + j] * si * (1 - 2 * x[j]);"),
    ("Tabu objective after the negation (reading S3)",
     "        dx[i] = -gi;\n        OV += gi;", "        dx[i] = -gi;\n        OV += dx[i];"),
    ("Tabu tenure one longer (reading S5)", "        C[i] += c;", "        C[i] += c + 1;"),
    ("Tabu memory decaying one step early",
     "            if (C[k] > 0)\n                C[k] -= 1;", "            if (C[k] > 1)\n                C[k] -= 1;"),
    ("Tabu ties to the highest index (reading S6)",
     "if (admissible && (i < 0 || dx[k] < dx[i]))", "if (admissible && (i < 0 || dx[k] <= dx[i]))"),
    ("Tabu keeping the last solution instead of the best visited (reading S7)",
     "    memcpy(x, xmin, (size_t)n);                        /* the search returns x_min */", ""),
    ("eta-hat scale 65535 instead of 2^16 (reading S9)",
     "(int32_t)((eta[j] * 65536) / mx)", "(int32_t)((eta[j] * 65535) / mx)"),
    ("gamma deviation |sum - z| instead of |2 sum - z| (Eq. 8)",
     "int64_t dev = 2 * col - z;", "int64_t dev = col - z;"),
    ("Delta as T / max T instead of 1 - T / max T (Eq. 7)",
     "(int32_t)((mx - T[j]) * 65536 / mx)", "(int32_t)(T[j] * 65536 / mx)"),
    ("Algorithm 3 adding w3 Delta instead of subtracting it",
     "w1 * eta_hat[j] + w2 * gamma[j] - w3 * delta[j]", "w1 * eta_hat[j] + w2 * gamma[j] + w3 * delta[j]"),
    ("Algorithm 3 truncating instead of flooring",
     "A[j] = (int32_t)orc_floor_div(v, 65536);", "A[j] = (int32_t)(v / 65536);"),
    ("Eq. 4 bias without the factor 2",
     "b += 2 * (int64_t)Q[(int64_t)S[a] * n + j] * x[j];", "b += (int64_t)Q[(int64_t)S[a] * n + j] * x[j];"),
    ("Eq. 4 bias summing over S as well",
     "            if (!in_s[j])\n                b += 2 *", "            if (1)\n                b += 2 *"),
    ("anneal local field without the factor 2",
     "field += 2 * (int64_t)Qs[(int64_t)pos * m + c] * xs[c];", "field += (int64_t)Qs[(int64_t)pos * m + c] * xs[c];"),
    ("anneal Metropolis test reversed (reading S14)",
     "(uint64_t)l * (uint64_t)beta[k] < (uint64_t)nlog[u >> 20]",
     "(uint64_t)l * (uint64_t)beta[k] > (uint64_t)nlog[u >> 20]"),
    ("anneal energy change not accumulated", "                dE += l;\n", "                dE += 0;\n"),
    ("exact IM minimising the wrong sign", "        if (f < best) { best = f; best_v = v; }",
     "        if (-f < best) { best = -f; best_v = v; }"),
    ("mutation probability reversed (reading S10)",
     "((uint64_t)((int64_t)A[i] - amin) * 4294967295ull)", "((uint64_t)((int64_t)amax - A[i]) * 4294967295ull)"),
    ("mutation candidates including S'", "        if (in_sel[i]) continue;\n", ""),
    ("Eq. 5 with period 16 instead of 15", "cos(M_PI * (double)t / 15.0)", "cos(M_PI * (double)t / 16.0)"),
    ("Eq. 5 without the 0.99^t decay", "* pow(0.99, (double)t);", "* pow(1.0, (double)t);"),
    ("cosine temperature schedule reversed",
     "(1.0 + cos(M_PI * (double)k / (double)(sweeps - 1))) / 2.0",
     "(1.0 - cos(M_PI * (double)k / (double)(sweeps - 1))) / 2.0"),
    ("Philox with a wrong Weyl constant", "k0 += 0x9E3779B9u;", "k0 += 0x9E3779BBu;"),
    ("Philox multiplier applied to the wrong word",
     "uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;", "uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c3;"),
    ("feature f4 = H / (t + 2) instead of H / (t + 1)",
     "f[4] = (float)((double)H[i] / (double)(t + 1));", "f[4] = (float)((double)H[i] / (double)(t + 2));"),
    ("feature f1 normalised by max |g| + 2 instead of max |g| + 1",
     "f[1] = (float)((double)g[i] / (double)(gmax + 1));", "f[1] = (float)((double)g[i] / (double)(gmax + 2));"),
    ("ranking by A ascending", "return orc_sort_key[i] > orc_sort_key[j] ? -1 : 1;",
     "return orc_sort_key[i] < orc_sort_key[j] ? -1 : 1;"),
    ("ranking ties to the highest index",
     "return orc_sort_key[i] > orc_sort_key[j] ? -1 : 1;\n    return i < j ? -1 : (i > j ? 1 : 0);",
     "return orc_sort_key[i] > orc_sort_key[j] ? -1 : 1;\n    return i > j ? -1 : (i < j ? 1 : 0);"),
    ("subQUBO groups not listed in ascending index order (reading S15)",
     "qsort(idx + off, (size_t)sizes[k], sizeof(int32_t), orc_cmp_int);", ""),
    ("best solution taking the last of equal energies", "if (E[p] < *best_E) {", "if (E[p] <= *best_E) {"),
    ("Jacobi and Gauss-Seidel bases swapped (reading S16)",
     "const uint8_t* base = prm->im_order == 1 ? x : S_pre;", "const uint8_t* base = prm->im_order == 1 ? S_pre : x;"),
    ("mutation subset size rounded up (reading S11)",
     "(int32_t)floor((double)(n - msel[p]) * r)", "(int32_t)ceil((double)(n - msel[p]) * r)"),
    ("network without the first ReLU", "h1[o] = a > 0.0f ? a : 0.0f;", "h1[o] = a;"),
    ("network without the output bias", "float s = W[ORC_B3];", "float s = 0.0f;"),
    ("score order with -0 equal to +0",
     "return -(int32_t)(b & 0x7FFFFFFFu) - 1;", "return -(int32_t)(b & 0x7FFFFFFFu);"),
    ("hit counts incremented twice",
     "if (H_io) H_io[(int64_t)p * n + idx[off + a]] += 1;", "if (H_io) H_io[(int64_t)p * n + idx[off + a]] += 2;"),
    ("Call_IM_Solution_Set one block short", "n / m;  /* No_IM", "n / m - 1;  /* No_IM"),
]


NET_SRC = os.path.join(ROOT, "oracle", "mlp_ref.py")

# the same for the double-precision network reference (oracle/mlp_ref.py),
# checked by the learned-selection pins
NET_MISTAKES = [
    ("ReLU derivative of the second layer dropped",
     "d2 = np.outer(ds, w3) * (a2 > 0)", "d2 = np.outer(ds, w3)"),
    ("first-layer backpropagation through W2 transposed",
     "d1 = (d2 @ W2) * (a1 > 0)", "d1 = (d2 @ W2.T) * (a1 > 0)"),
    ("output bias gradient averaged twice", "gb3 = ds.sum()", "gb3 = ds.mean()"),
    ("loss derivative with the wrong sign on positives",
     "ds = (pos_weight * y * (sg - 1.0) + (1.0 - y) * sg) / B",
     "ds = (pos_weight * y * (1.0 - sg) + (1.0 - y) * sg) / B"),
    ("positive-class weight applied to the negatives",
     "ds = (pos_weight * y * (sg - 1.0) + (1.0 - y) * sg) / B",
     "ds = (y * (sg - 1.0) + pos_weight * (1.0 - y) * sg) / B"),
    ("loss derivative not divided by the batch",
     "ds = (pos_weight * y * (sg - 1.0) + (1.0 - y) * sg) / B",
     "ds = (pos_weight * y * (sg - 1.0) + (1.0 - y) * sg)"),
    ("second-layer bias missing in the forward pass", "a2 = h1 @ W2.T + b2", "a2 = h1 @ W2.T"),
    ("softplus without its stable branch", "np.log1p(np.exp(-np.abs(v)))", "np.log1p(np.exp(-v))"),
    ("sigmoid at twice the slope", "0.5 * (1.0 + np.tanh(0.5 * v))", "0.5 * (1.0 + np.tanh(v))"),
    ("Adam without the first-moment bias correction", "mh = m / (1.0 - beta1 ** step)", "mh = m"),
    ("Adam second moment of |g| instead of g^2", "(1.0 - beta2) * g * g", "(1.0 - beta2) * np.abs(g)"),
    ("BF16 rounding with ties away from zero",
     "((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16", "((b + 0x8000) >> 16) << 16"),
]

PLUGIN = """import importlib.util, os, sys
_spec = importlib.util.spec_from_file_location("oracle.mlp_ref", os.path.join(os.path.dirname(__file__), "mlp_ref.py"))
_mod = importlib.util.module_from_spec(_spec)
_spec.loader.exec_module(_mod)
sys.modules["oracle.mlp_ref"] = _mod
"""


def _net_pins(src_text, out_dir):
    os.makedirs(out_dir)
    with open(os.path.join(out_dir, "mlp_ref.py"), "w") as f:
        f.write(src_text)
    with open(os.path.join(out_dir, "planted_netref.py"), "w") as f:
        f.write(PLUGIN)
    env = dict(os.environ, PYTHONPATH=out_dir + os.pathsep + os.environ.get("PYTHONPATH", ""))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "-p", "planted_netref",
                        "tests/test_oracle_learned.py"], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=600)
    return r.returncode, r.stdout[-2000:]


def _build(src_text, out_dir, name):
    src = os.path.join(out_dir, name + ".c")
    lib = os.path.join(out_dir, name + ".so")
    with open(src, "w") as f:
        f.write(src_text)
    subprocess.run(["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off", "-fPIC", "-shared", "-o", lib,
                    src, "-lm"], check=True, capture_output=True)
    return lib


def _pins(lib):
    env = dict(os.environ, ICD2S_ORACLE_LIB=lib)
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", *PINS],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return r.returncode, r.stdout[-2000:]


def test_planted_mistakes_fail_a_pin(tmp_path):
    text = open(SRC).read()
    for what, old, new in MISTAKES:
        assert text.count(old) == 1, "the oracle changed near: " + what
    rc, out = _pins(_build(text, str(tmp_path), "unchanged"))
    assert rc == 0, out

    def one(k):
        what, old, new = MISTAKES[k]
        lib = _build(text.replace(old, new), str(tmp_path), "mistake%02d" % k)
        return what, _pins(lib)

    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 2)) as ex:
        results = list(ex.map(one, range(len(MISTAKES))))
    missed = [what for what, (rc, _) in results if rc == 0]
    errors = [(what, out) for what, (rc, out) in results if rc not in (0, 1)]
    assert not errors, errors
    assert not missed, "no pin fails with: " + "; ".join(missed)


def test_planted_mistakes_in_the_network_reference_fail_a_pin(tmp_path):
    text = open(NET_SRC).read()
    for what, old, new in NET_MISTAKES:
        assert text.count(old) == 1, "the network reference changed near: " + what
    rc, out = _net_pins(text, str(tmp_path / "unchanged"))
    assert rc == 0, out

    def one(k):
        what, old, new = NET_MISTAKES[k]
        return what, _net_pins(text.replace(old, new), str(tmp_path / ("mistake%02d" % k)))

    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 2)) as ex:
        results = list(ex.map(one, range(len(NET_MISTAKES))))
    missed = [what for what, (rc, _) in results if rc == 0]
    errors = [(what, out) for what, (rc, out) in results if rc not in (0, 1)]
    assert not errors, errors
    assert not missed, "no pin fails with: " + "; ".join(missed)
