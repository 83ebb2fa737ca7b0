"""Host-side arithmetic of bench.py: the roofline object's counts and the
per-step flop model (no GPU)."""
import math
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _stage(rr_ms):
    return {"resid": 3.0, "hpsi": 80.0, "gram": 19.0, "rr": sum(rr_ms.values()), "rot": 22.0}


def test_hemv_slice_bytes():
    import bench
    # below the threshold every Hermitian product runs on the FP64 pipe
    assert bench.hemv_slice_bytes(1024) == 0
    # order 1025: one panel (columns 0..31, trailing order 1024); nine
    # 128-row tile rows, 45 lower tiles of 512 KB read per column
    assert bench.hemv_slice_bytes(1025) == 32 * 45 * 512 * 1024
    # order 1200: panels at 0, 32, ..., 160 (trailing order >= 1024); ten
    # tile rows; columns 127..191 start at tile 1 (45 tiles), the rest at
    # tile 0 (55 tiles)
    assert bench.hemv_slice_bytes(1200) == (127 * 55 + 65 * 45) * 512 * 1024
    # roughly 16 bytes per real entry of the lower triangle per column
    n = 3456
    assert 0.8 < bench.hemv_slice_bytes(n) / (32 * n ** 3 / 6) < 1.3


def test_roofline_tensor_stage_counts():
    import bench
    n, nb, npw = 3456, 1152, 104415
    rr = {"chol_inv": 1.0, "transform": 60.0, "tridiag": 2.0, "dc": 0.5, "backtransform": 1.0}
    fl = bench.step_flops(npw, nb, n, nb, 2048, (96, 96, 96), hcols=n)
    roof = bench.roofline(_stage(rr) | {"hpsi": 0.1, "gram": 19.0, "rot": 22.0, "resid": 0.1}, rr, fl, n, nb,
                          "mixed")
    peak = bench.measured_peaks().get("bf16_tflops_sustained")
    if peak:
        # the split-FP16 GEMM over its three stages: S^H S (Hermitian half,
        # 4 npw n^2), S M and H S M (triangular M: half of 8 npw n^2 each) and
        # S~^H H S~ (Hermitian half), the rotations S~ Y and S C_P (C_P's
        # first nb rows zero); three split-FP16 slice products each
        t_gram = 4.0 * npw * n * n
        t_tr = 2 * 4.0 * npw * n * n + 4.0 * npw * n * n
        t_rot = 8.0 * npw * n * nb + 8.0 * npw * (n - nb) * nb
        assert roof["stage"] == "tc_gemm" and roof["bound"] == "tensor"
        assert math.isclose(roof["ms"], 19.0 + 60.0 + 22.0)
        assert math.isclose(roof["achieved"], 3 * (t_gram + t_tr + t_rot) / 101e-3 / 1e12, rel_tol=1e-12)
        assert math.isclose(roof["frac"], roof["achieved"] / peak, rel_tol=1e-12)
        g = roof["stages"]["tc_gemm_gram"]
        assert math.isclose(g["tensor_tflops"], 3 * t_gram / 19e-3 / 1e12, rel_tol=1e-12)
    hbm = bench.measured_peaks().get("hbm_gbs")
    if hbm:
        h = roof["stages"]["householder"]
        assert math.isclose(h["achieved_gbs"], bench.hemv_slice_bytes(n) / 2e-3 / 1e9, rel_tol=1e-12)


def test_step_flops_model():
    import bench
    npw, nb, ns, nproj, grid = 1000, 10, 30, 40, (16, 16, 16)
    f = bench.step_flops(npw, nb, ns, nb, nproj, grid)
    n3 = 16 ** 3
    assert math.isclose(f["fft"], 2 * 5.0 * n3 * math.log2(n3) * nb)
    assert f["proj"] == 2 * 8.0 * npw * nproj * nb
    assert f["gram"] == 2 * 4.0 * npw * ns * ns
    assert f["rot"] == 2 * 8.0 * npw * nb * (ns - nb) + 2 * 8.0 * npw * nb * nb
    # H applied to X, W and P in mixed precision
    g = bench.step_flops(npw, nb, ns, nb, nproj, grid, hcols=ns)
    assert math.isclose(g["fft"] / f["fft"], ns / nb)


def test_cpu_baseline_sample_is_stated_as_extrapolated():
    # the oracle's sampled step (small workload): every piece carries its
    # measured seconds and its scale, the step is their scaled sum
    import bench
    sec, note, parts = bench.oracle_sample(bench.WORKLOADS["si8"])
    assert set(parts) == {"hpsi", "gram", "rot", "rr"}
    for p in parts.values():
        assert p["measured_s"] > 0 and p["scale"] >= 1
        assert math.isclose(p["scaled_s"], p["measured_s"] * p["scale"], rel_tol=1e-12)
    assert math.isclose(sec, sum(p["scaled_s"] for p in parts.values()), rel_tol=1e-12)
    assert "scaled" in note
