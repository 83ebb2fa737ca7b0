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


def test_roofline_dominant_fp64_stage():
    import bench
    n, nb = 3456, 1152
    rr = {"chol_inv": 41.0, "transform": 60.0, "tridiag": 204.0, "dc": 47.0, "backtransform": 25.0}
    fl = bench.step_flops(104415, nb, n, nb, 2048, (96, 96, 96), hcols=n)
    roof = bench.roofline(_stage(rr), rr, fl, n, nb, "mixed")
    assert roof["stage"] == "tridiag" and roof["bound"] == "alu"
    # FP64-ALU work of the Householder reduction: the Hermitian products,
    # sum_c 8 (n - c)^2 = 8 n^3 / 3 flop, over the stage's time
    ach = 8 * n ** 3 / 3 / 0.204 / 1e12
    assert math.isclose(roof["achieved"], ach, rel_tol=1e-12)
    assert math.isclose(roof["frac"], ach / bench.FP64_PEAK_TFLOPS, rel_tol=1e-12)
    assert roof["unit"] == "TFLOP/s" and roof["ms"] == 204.0
    # DRAM traffic of the reduction, scaled from the one-kernel capture
    assert math.isclose(roof["traffic"], 16.73 * n ** 3 / 6)
    other = bench.roofline(_stage(rr), rr, fl, 3000, nb, "mixed")
    assert other["traffic"] is None
    st = roof["stages"]
    assert math.isclose(st["householder_fp64"]["frac"], roof["frac"])


def test_roofline_tensor_stage_counts():
    import bench
    n, nb, npw = 3456, 1152, 104415
    rr = {"chol_inv": 1.0, "transform": 60.0, "tridiag": 2.0, "dc": 0.5, "backtransform": 1.0}
    fl = bench.step_flops(npw, nb, n, nb, 2048, (96, 96, 96), hcols=n)
    roof = bench.roofline(_stage(rr) | {"hpsi": 0.1, "gram": 19.0, "rot": 22.0, "resid": 0.1}, rr, fl, n, nb,
                          "mixed")
    assert roof["stage"] == "transform"
    peak = bench.measured_peaks().get("bf16_tflops_sustained")
    if peak:
        # S M and H S M (triangular M: half of 8 npw n^2 each) and S~^H H S~
        # (Hermitian half), three split-FP16 slice products each
        t = 3 * (2 * 4.0 * npw * n * n + 4.0 * npw * n * n)
        assert roof["bound"] == "tensor"
        assert math.isclose(roof["achieved"], t / 60e-3 / 1e12, rel_tol=1e-12)
        g = roof["stages"]["tc_gemm_gram"]
        assert math.isclose(g["tensor_tflops"], 3 * 4.0 * npw * n * n / 19e-3 / 1e12, rel_tol=1e-12)


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
