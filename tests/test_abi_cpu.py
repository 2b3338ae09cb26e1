"""The C-ABI library without a GPU: it builds for sm_103a, loads, exports
every entry point that include/icd2s.h declares, computes its host tables
exactly as the oracle does, and rejects bad arguments before touching CUDA."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2502_13947_gb300 import build as B
from paper_2502_13947_gb300 import icd2s as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "icd2s.h")


@pytest.fixture(scope="module")
def built():
    B.build()
    return I.lib()


def declared_entry_points():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:const char\*|int32_t|int)\s+(icd2s_\w+)\s*\(", src, re.M)))


def test_header_and_binding_agree():
    assert declared_entry_points() == sorted(I.EXPORTS)


def test_library_exports_every_declared_symbol(built):
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (icd2s_\w+)", out))
    missing = set(declared_entry_points()) - exported
    assert not missing, missing
    for name in declared_entry_points():
        assert hasattr(built, name)


def test_library_targets_sm_103a_only():
    """The build passes one -gencode, sm_103a machine code with no other
    target, to every nvcc command (compile and link)."""
    assert B.ARCH == "-gencode=arch=compute_103a,code=sm_103a"
    src = open(B.__file__).read()
    assert set(re.findall(r"(?:compute|sm)_\d+a?", src)) == {"compute_103a", "sm_103a"}
    assert src.count("[nvcc, *common,") == 1 and "common = [ARCH," in src
    assert src.count("[nvcc, ARCH, \"-shared\"") == 1


def test_host_tables_equal_the_oracles(built, orc):
    for sweeps, tmax, tmin in [(1, 50.0, 2.0), (7, 100.0, 1.0), (256, 812.5, 0.75), (1024, 3000.0, 1.0)]:
        b, t = I.icd2s_tables(sweeps, tmax, tmin)
        assert np.array_equal(b, orc.beta_table(sweeps, tmax, tmin))
        assert np.array_equal(t, orc.nlog_table())


def test_default_params_follow_table_1(built):
    p = I.icd2s_default_params(2500)
    assert (p.z, p.alpha, p.c, p.w1, p.w2, p.w3, p.m_max, p.K) == (4, 12500, 16, 65536, 65536, 32768, 50, 1)
    p = I.icd2s_default_params(64)
    assert p.c == 2 and p.m_max == 50 and p.alpha == 320
    assert I.icd2s_default_params(3).m_max == 3


def test_argument_errors_are_reported_without_a_gpu(built):
    with pytest.raises(I.ICD2SError) as e:
        I.icd2s_default_params(0)
    assert e.value.code == I.ERR_RANGE and "n=0" in str(e.value)
    L = built
    h = ctypes.c_void_p()
    assert L.icd2s_qubo_create(None, 5, ctypes.byref(h)) == I.ERR_ARG
    Q = np.zeros((4, 4), np.int8)
    assert L.icd2s_qubo_create(Q.ctypes.data_as(ctypes.c_void_p), 20000, ctypes.byref(h)) == I.ERR_RANGE
    assert b"n=20000" in L.icd2s_last_error()
    assert L.icd2s_state_create(None, 4, 1, ctypes.byref(h)) == I.ERR_ARG
    assert L.icd2s_tabu(None, 10, 2, None) == I.ERR_ARG
    assert L.icd2s_qubo_destroy(None) == I.OK and L.icd2s_state_destroy(None) == I.OK


def test_forced_allocation_failure_is_reported_without_a_gpu(built):
    """With the allocation hook at 0 the first device allocation of
    icd2s_qubo_create fails before any CUDA call: ICD2S_ERR_OOM, no handle."""
    Q = np.zeros((8, 8), np.int8)
    h = ctypes.c_void_p(1)
    I.icd2s_debug_fail_allocations_after(0)
    try:
        assert built.icd2s_qubo_create(Q.ctypes.data_as(ctypes.c_void_p), 8, ctypes.byref(h)) == I.ERR_OOM
    finally:
        I.icd2s_debug_fail_allocations_after(-1)
    assert not h.value and b"allocation" in built.icd2s_last_error()


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    monkeypatch.setattr(I, "LIB_PATH", str(tmp_path / "nope.so"))
    monkeypatch.setattr(I, "_lib", None)
    with pytest.raises(I.ICD2SError) as e:
        I.icd2s_version()
    assert "missing" in str(e.value)


def test_struct_layouts_match_the_header(tmp_path):
    """sizeof/offsetof of every parameter struct, from a C probe compiled
    against the header, equal the ctypes mirrors of the binding."""
    structs = {"icd2s_params": I.Params, "icd2s_anneal_params": I.AnnealParams,
               "icd2s_select_params": I.SelectParams, "icd2s_mutate_params": I.MutateParams,
               "icd2s_stats": I.Stats, "icd2s_tuning": I.Tuning, "icd2s_train_params": I.TrainParams}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "icd2s.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append('printf("%s size %%zu\\n", sizeof(%s));' % (cname, cname))
        for f, _ in py._fields_:
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (cname, f, cname, f))
    lines.append("return 0; }")
    src = tmp_path / "probe.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "probe"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.run(["gcc", "-std=c11", "-I", inc, str(src), "-o", str(exe)], check=True)
    got = dict(l.rsplit(" ", 1) for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                         check=True).stdout.splitlines())
    for cname, py in structs.items():
        assert int(got["%s size" % cname]) == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert int(got["%s %s" % (cname, f)]) == getattr(py, f).offset, (cname, f)
