"""Host-side checks of libheom that need no GPU: the library loads, exports every function that
include/heom.h declares, builds the hierarchy bit-exactly like the oracle, and rejects bad
arguments with the documented error codes."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle.oracle import hier_export
from paper_1803_03498_gb300 import heom
from paper_1803_03498_gb300 import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1803_03498_gb300.build import build
    build()
    return heom.load()


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "heom.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(heom_[a-z0-9_]+)\s*\(", txt)))


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(names) == sorted(heom.ABI_SYMBOLS)


@pytest.mark.parametrize("M", range(1, 9))
@pytest.mark.parametrize("D", range(0, 7))
def test_hierarchy_bit_exact_small(lib, M, D):
    h = heom.Hierarchy(M, D)
    t, p, m = h.export()
    to, po, mo = hier_export(M, D)
    assert np.array_equal(t, to) and np.array_equal(p, po) and np.array_equal(m, mo)


@pytest.mark.parametrize("M,D", [(2, 4), (14, 4), (28, 6)])
def test_hierarchy_bit_exact_workloads(lib, M, D):
    h = heom.Hierarchy(M, D)
    t, p, m = h.export()
    to, po, mo = hier_export(M, D)
    assert t.tobytes() == to.tobytes()
    assert p.tobytes() == po.tobytes()
    assert m.tobytes() == mo.tobytes()
    from math import comb
    assert list(h.level_offsets) == [0] + [comb(M + L - 1, M) for L in range(1, D + 2)]


def test_hierarchy_errors(lib):
    for M, D, code in [(0, 2, heom.HEOM_E_ARG), (3, -1, heom.HEOM_E_ARG), (256, 1, heom.HEOM_E_ARG),
                       (200, 10, heom.HEOM_E_OVERFLOW)]:
        with pytest.raises(heom.HeomError) as ei:
            heom.Hierarchy(M, D)
        assert ei.value.code == code


def test_run_bytes_and_argument_errors(lib):
    p = wl.dimer()
    h = heom.Hierarchy(p.system.n_modes, p.system.D)
    b64 = heom.run_bytes(p.system, h, "fp64", 10)
    b32 = heom.run_bytes(p.system, h, "fp32_mixed", 10)
    # the split-TF32 precision stores exactly what the mixed precision stores
    assert heom.run_bytes(p.system, h, "split_tf32", 10) == b32
    assert b64 > 0 and b32 > 0
    big = wl.lhcii_like().system
    hb = heom.Hierarchy(big.n_modes, big.D)
    n_ado, E = hb.n_ado, 14 * 14
    assert heom.run_bytes(big, hb, "fp64", 1) >= 3 * n_ado * E * 16
    assert heom.run_bytes(big, hb, "fp32_mixed", 1) >= 3 * n_ado * E * 8
    assert heom.run_bytes(big, hb, "fp32_mixed", 1) < 3 * n_ado * E * 12
    # mode count mismatch
    with pytest.raises(heom.HeomError) as ei:
        heom.run_bytes(p.system, heom.Hierarchy(3, 2), "fp64", 1)
    assert ei.value.code == heom.HEOM_E_ARG
    # unknown precision
    sa = heom._SysArgs(p.system)
    out = ctypes.c_size_t()
    assert lib.heom_run_bytes(ctypes.byref(sa.s), h._h, 7, 1, ctypes.byref(out)) == heom.HEOM_E_ARG
    # bath state out of range
    bad = wl.System("bad", p.system.H, [0, 5], [35.0] * 2, [50.0] * 2, [300.0] * 2, K=0, D=4)
    with pytest.raises(heom.HeomError):
        heom.run_bytes(bad, h, "fp64", 1)
    # too many states (the general kernel covers up to 32)
    H = np.eye(33)
    bad = wl.System("big", H, [0], [35.0], [50.0], [300.0], K=0, D=1)
    with pytest.raises(heom.HeomError):
        heom.run_bytes(bad, heom.Hierarchy(1, 1), "fp64", 1)
    assert "n_states" in lib.heom_last_error().decode()


def test_schedule_candidates_and_autotune_switch(lib):
    """The tuner's candidate sets (host only) and the process-wide switch."""
    assert heom.schedule_candidates(0) == [(100, 1), (75, 1), (50, 1)]
    both = [(100, 1), (50, 1), (100, 2), (50, 2), (100, 4), (50, 4)]
    assert heom.schedule_candidates(1) == both and heom.schedule_candidates(2) == both
    with pytest.raises(heom.HeomError) as ei:
        heom.schedule_candidates(3)
    assert ei.value.code == heom.HEOM_E_ARG
    prev = heom.set_autotune(-1)  # query
    assert prev >= 0
    assert heom.set_autotune(5) == prev
    assert heom.set_autotune(-1) == 5
    heom.set_autotune(prev)
    heom.tune_cache_clear()
    heom.set_default_schedule(1, (50, 4))
    heom.set_default_schedule(1, None)
    with pytest.raises(heom.HeomError) as ei:
        heom.set_default_schedule(0, (100, 3))
    assert ei.value.code == heom.HEOM_E_ARG


def test_general_runs_bytes_and_mask_checks(lib):
    """Runs on the general kernel: the records per link grow with the states of each V_b, a fourth
    state copy is reserved for time-dependent runs, and bath_mask entries are checked."""
    prop, _ = wl.fmo_two_exciton(n_sites=4, D=2)
    s = prop.system
    h = heom.Hierarchy(s.n_modes, s.D)
    assert s.N == 11
    b3 = heom.run_bytes(s, h, "fp64", 4)
    b4 = heom.run_bytes(s, h, "fp64", 4, time_dependent=True)
    assert b4 - b3 >= h.n_ado * s.N * s.N * 16  # one more FP64 copy
    plain = wl.System("no mask", s.H, s.bath_state, s.lambda_cm, s.tau_fs, s.T_K, K=s.K, D=s.D)
    # each site's V has 1 + 3 states here (its single and the three pairs with it): 4 records per link
    links = int(np.sum(h.export()[1] >= 0) + np.sum(h.export()[2] >= 0))
    assert b3 - heom.run_bytes(plain, h, "fp64", 4) >= 3 * links * 32
    bad = wl.System("bad", s.H, s.bath_state, s.lambda_cm, s.tau_fs, s.T_K, K=s.K, D=s.D,
                    bath_mask=np.full_like(s.bath_mask, 2))
    with pytest.raises(heom.HeomError) as ei:
        heom.run_bytes(bad, h, "fp64", 1)
    assert ei.value.code == heom.HEOM_E_ARG and "bath_mask" in lib.heom_last_error().decode()
    g7, _ = wl.fmo_two_exciton(n_sites=7, D=1)
    assert g7.system.N == 29
    heom.run_bytes(g7.system, heom.Hierarchy(g7.system.n_modes, 1), "fp32_mixed", 1)


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """No CPU fallback: without libheom.so the binding raises instead of computing anything."""
    monkeypatch.setattr(heom, "_lib", None)
    monkeypatch.setattr(heom, "LIB_PATH", str(tmp_path / "libheom.so"))
    with pytest.raises(RuntimeError, match="libheom.so not found"):
        heom.load()
    with pytest.raises(RuntimeError):
        heom.Hierarchy(2, 2)
