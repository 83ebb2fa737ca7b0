"""The C-ABI library loads and exports every entry point include/pw.h declares
(no compute calls: runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(pw_\w+)\s*\(", txt))
    return sorted(names)


def test_header_declares_the_boundary():
    names = _declared()
    for n in ["pw_setup_cell", "pw_apply_H", "pw_subspace_step", "pw_eigsolve", "pw_strerror",
              "pw_destroy_cell", "pw_cell_info"]:
        assert n in names


def test_library_exports_every_symbol():
    import __graft_entry__
    lib_path = __graft_entry__._build_module().build()
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_strerror_without_gpu():
    import paper_2406_10765_gb300 as pw
    assert pw.pw_strerror(0) == "ok"
    assert "positive definite" in pw.pw_strerror(-4)


def test_autotuner_host_entry_points_without_gpu():
    # the plan table and the GEMM tuning switch need no device
    import paper_2406_10765_gb300 as pw
    for n in (16, 24, 32, 36, 48, 64, 72, 96, 128, 144):
        plans = pw.pw_fft_plans(n)
        assert plans, n
        assert len(set(plans)) == len(plans)
        for L, R in plans:
            assert L * R == n and L & (L - 1) == 0 and 1 <= L <= 32 and R <= 18
    assert pw.pw_fft_plans(27) == [] and pw.pw_fft_plans(0) == []
    with pytest.raises(pw.PwError):
        pw.pw_autotune_gemm(3)
    with pytest.raises(pw.PwError):
        pw.pw_autotune_gemm(2, 0)
    pw.pw_autotune_gemm(2, 4)
    pw.pw_autotune_gemm(0)
    assert pw.pw_autotune_gemm_table() == ""


def test_gemm_tuning_table_round_trip_without_gpu():
    # a saved K-split table loads back into the process-wide table unchanged
    import paper_2406_10765_gb300 as pw
    pw.pw_autotune_gemm(0)
    saved = ("mtiles=18 ntiles=9 k<=262144 k_lo=0 tri_b=0 herm=1 mode=0 split=8 ms1=2.6580 ms=1.7670\n"
             "mtiles=2 ntiles=18 k<=4096 k_lo=128 tri_b=1 herm=0 mode=1 split=3 ms1=0.5000 ms=0.2500\n")
    assert pw.pw_autotune_gemm_load(saved) == 2
    table = pw.pw_autotune_gemm_table()
    assert sorted(table.splitlines()) == sorted(saved.splitlines())
    with pytest.raises(pw.PwError):
        pw.pw_autotune_gemm_load("mtiles=1 ntiles=1 k<=100 k_lo=0 tri_b=0 herm=0 mode=0 split=2 ms1=1 ms=1\n")
    # a dump whose last line is malformed adds none of its good lines
    bad = ("mtiles=5 ntiles=5 k<=4096 k_lo=0 tri_b=0 herm=0 mode=0 split=4 ms1=1.0000 ms=0.5000\n"
           "mtiles=5 ntiles=6 k<=4096 k_lo=0 tri_b=0 herm=0 mode=0 split=99 ms1=1.0000 ms=0.5000\n")
    with pytest.raises(pw.PwError):
        pw.pw_autotune_gemm_load(bad)
    assert sorted(pw.pw_autotune_gemm_table().splitlines()) == sorted(saved.splitlines())
    pw.pw_autotune_gemm(0)
    assert pw.pw_autotune_gemm_table() == ""
