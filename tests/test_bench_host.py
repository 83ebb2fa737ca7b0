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
    rr = {"chol_inv": 143.0, "transform": 60.0, "tridiag": 295.0, "dc": 47.0, "backtransform": 160.0}
    fl = bench.step_flops(104415, nb, n, nb, 2048, (96, 96, 96), hcols=n)
    roof = bench.roofline(_stage(rr), rr, fl, n, nb, "mixed")
    assert roof["stage"] == "tridiag" and roof["bound"] == "alu"
    # Householder reduction: 16 n^3 / 3 flop over the stage's time
    ach = 16 * n ** 3 / 3 / 0.295 / 1e12
    assert math.isclose(roof["achieved"], ach, rel_tol=1e-12)
    assert math.isclose(roof["frac"], ach / bench.FP64_PEAK_TFLOPS, rel_tol=1e-12)
    assert roof["unit"] == "TFLOP/s" and roof["ms"] == 295.0
    # the FP64 Rayleigh-Ritz parts of the mixed path (the transform runs on tensor cores)
    assert roof["rr_fp64"]["parts"] == ["backtransform", "chol_inv", "tridiag"]
    assert math.isclose(roof["rr_fp64"]["ms"], 295.0 + 143.0 + 160.0)
    # DRAM traffic only for the captured configuration
    assert roof["traffic"] == bench.NCU_TRAFFIC[("tridiag", n, nb)][0]
    other = bench.roofline(_stage(rr), rr, fl, 3000, nb, "mixed")
    assert other["traffic"] is None


def test_roofline_fp64_transform_counts():
    import bench
    n, nb = 432, 144
    rr = {"chol_inv": 1.0, "transform": 9.0, "tridiag": 2.0, "dc": 0.5, "backtransform": 1.0}
    fl = bench.step_flops(13056, nb, n, nb, 256, (48, 48, 48))
    roof = bench.roofline(_stage(rr) | {"hpsi": 0.1, "gram": 0.1, "rot": 0.1, "resid": 0.1}, rr, fl, n, nb,
                          "fp64")
    assert roof["stage"] == "transform"
    assert math.isclose(roof["achieved"], 8.0 * n ** 3 / 9e-3 / 1e12, rel_tol=1e-12)
    assert "transform" in roof["rr_fp64"]["parts"]


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
