#!/usr/bin/env python3
"""Benchmark: LOBPCG block-eigensolver steps per second on the synthetic Si
512-atom supercell (4x4x4 diamond cells, a = 10.26 bohr, Ecut = 10 Ha,
npw = 104,415, grid 96^3, 1152 bands, 2048 KB projectors), one step = one
pass of the whole hot path: residual + preconditioner, H W (FFT local term +
projector contractions), S^H S and S^H H S, FP64 Rayleigh-Ritz (Cholesky,
L^-1, Hermitian eigensolve), rotations.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64|mixed]
  python bench.py --impl reference      # the FP64 CPU oracle on a bounded sample

Prints one JSON line (rank 0).  Multi-GPU runs are independent replicas
(weak scaling); only the timing is reduced across ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "si512": dict(species="Si", n=4, ecut=10.0, nb=1152,
                  name="Si-512 (4x4x4 diamond cells, a=10.26 bohr), Gamma, Ecut=10 Ha"),
    "si8": dict(species="Si", n=1, ecut=10.0, nb=24,
                name="Si-8 (diamond cell, a=10.26 bohr), Gamma, Ecut=10 Ha"),
    "si1728": dict(species="Si", n=6, ecut=8.0, nb=3840, onthefly=True,
                   name="Si-1728 (6x6x6 diamond cells, a=10.26 bohr), Gamma, Ecut=8 Ha"),
}
E2E_STEPS = 20                      # e2e: full steps (tol 0, no locking) through pw_eigsolve
SOLVE_TOL, SOLVE_MAXIT = 5e-6, 200  # time to solution (Si-512 mixed converges in ~120 steps)
REF_TOL, REF_MAXIT = 5e-7, 80       # FP64 reference solve started from the mixed result
DEPS_TARGET = 1e-6                  # |delta eps| of the metric, Ha
# Householder reduction: panels of 32 columns whose trailing order is at
# least this run their Hermitian products on the tensor cores
HS_MIN_ORDER = 1024
FP64_PEAK_TFLOPS = 1.25     # nominal FP64 rate of the part (no FP64 tensor path)
FP32_PEAK_TFLOPS = 80.5     # nominal FP32 rate: 152 SMs x 128 lanes x 2 x 2.07 GHz
METRIC = "Si-512 eigensolver iters/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 comparison step")
    ap.add_argument("--workload", default="si512", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=E2E_STEPS,
                    help="full steps of the end-to-end pw_eigsolve call")
    ap.add_argument("--no-accuracy", action="store_true",
                    help="skip the solve to tolerance and its FP64 reference (|delta eps|)")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-si1728", action="store_true",
                    help="skip the Si-1728 step measured after the Si-512 line's work")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default FFT plan and K split instead of the autotuner's")
    ap.add_argument("--serve-requests", type=int, default=32,
                    help="requests per arrival rate (a prefix of the seeded 2000-request stream)")
    ap.add_argument("--serve-rates", default="0.5,1,2",
                    help="Poisson arrival rates (requests/s) of the serving sweep")
    ap.add_argument("--serve-slots", type=int, default=4)
    ap.add_argument("--serve-only", action="store_true",
                    help="run only the serving sweep and print its line")
    return ap.parse_args()


def serve_sweep(args):
    """Served fixed-potential eigensolves at several Poisson arrival rates:
    for each rate the first N requests of the seeded 2000-request stream
    (Si/C diamond cells, n in 1..3, Ecut ~ U[8, 12] Ha, bands = 1.125 x
    occupied), continuous batching in mixed precision: solves/s over the
    wall time and p50/p99 latency (arrival to result)."""
    import numpy as np
    import synth
    import paper_2406_10765_gb300 as pw
    out = []
    for rate in [float(x) for x in args.serve_rates.split(",") if x]:
        reqs = synth.serving_requests(2000, rate_per_s=rate, seed=2024)[:args.serve_requests]
        t0 = time.perf_counter()
        res = pw.pw_serve(reqs, max_slots=args.serve_slots, precision="mixed", autotune=not args.no_autotune)
        wall = time.perf_counter() - t0
        ok = [o for o in res if o["status"] in (0, -5)]
        lat = np.array([o["latency"] for o in ok])
        out.append({"arrival_rate_per_s": rate, "requests": len(reqs), "completed": len(ok),
                    "converged": sum(o["status"] == 0 for o in res),
                    "status_counts": {str(k): sum(o["status"] == k for o in res)
                                      for k in sorted(set(o["status"] for o in res))},
                    "solves_per_s": len(ok) / wall, "wall_s": wall,
                    "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
                    "max_resid": float(max(o["max_resid"] for o in ok)),
                    "last_arrival_s": float(reqs[-1]["t_arrival"])})
    return {"metric": "served fixed-potential eigensolves", "slots": args.serve_slots, "precision": "mixed",
            "autotune": not args.no_autotune, "rates": out,
            "sample": f"first {args.serve_requests} requests of the seeded 2000-request stream at each rate"}


def accuracy_run(pw, torch, cell, nb, x0, barrier):
    """The metric's accuracy condition: a mixed-precision solve to SOLVE_TOL
    (step by step, Ritz values after every step), its FP64 polish, then an
    FP64 solve to REF_TOL started from the mixed block as the reference.
    Reports max |eps_mixed - eps_fp64| and the time and steps the mixed solve
    took to bring every Ritz value within DEPS_TARGET of the reference."""
    import numpy as np
    barrier()
    t0 = time.perf_counter()
    s = pw.pw_solver_create(cell.h, nb, tol=SOLVE_TOL, x0=x0, precision="mixed")
    hist, it = [], 0
    while True:
        e, r = pw.pw_solver_eigs(s, nb)
        hist.append((time.perf_counter() - t0, it, e.copy()))
        if r.max() <= SOLVE_TOL or it >= SOLVE_MAXIT:
            break
        rep = pw.pw_subspace_step(cell.h, s)
        it += 1
        if rep.nactive == 0:
            break
    pw.pw_solver_polish(s)
    e_mix, r_mix = pw.pw_solver_eigs(s, nb)
    t_mix = time.perf_counter() - t0
    psi = pw.new_block(cell.npw, nb)
    pw.pw_solver_block(s, psi)
    pw.pw_solver_destroy(s)
    cell.set_precision("fp64")
    barrier()
    t1 = time.perf_counter()
    e_ref, rep64, st64 = pw.pw_eigsolve(cell.h, nb, tol=REF_TOL, maxit=REF_MAXIT, x0=psi, precision="fp64",
                                        raise_noconv=False)
    barrier()
    t_ref = time.perf_counter() - t1
    cell.set_precision("mixed")
    reach = next(((t, k) for (t, k, e) in hist if np.abs(e - e_ref).max() <= DEPS_TARGET), None)
    deps = float(np.abs(e_mix - e_ref).max())
    return {"max_abs_deps": deps, "deps_target": DEPS_TARGET, "met": deps <= DEPS_TARGET,
            "mixed_solve": {"tol": SOLVE_TOL, "steps": it, "seconds": t_mix, "max_resid_fp64": float(r_mix.max()),
                            "solves_per_s": 1.0 / t_mix},
            "reach_deps_target": {"seconds": reach[0], "steps": reach[1]} if reach else None,
            "fp64_reference": {"tol": REF_TOL, "steps": rep64.iters, "seconds": t_ref,
                               "max_resid": rep64.max_resid, "status": int(st64),
                               "orth_err": rep64.orth_err},
            "note": "mixed solve from the seeded start to max residual <= tol, then its FP64 Rayleigh-Ritz "
                    "polish; reference: FP64 LOBPCG from the mixed block to max residual <= 5e-7 (each "
                    "reference value within its residual of an exact eigenvalue); reach = first step whose "
                    "Ritz values are all within the target of the reference"}


def si1728_step(pw, torch, args):
    """One mixed LOBPCG step of the 1,728-atom cell (Ecut 8 Ha, npw 251,967,
    grid 128^3, 3,840 bands, 6,912 projectors generated on the fly, tall
    products in plane-wave chunks), timed with CUDA events after one warm-up
    step: the steady step with P (Rayleigh-Ritz order 11,520)."""
    import gc
    import numpy as np
    import synth
    gc.collect()
    torch.cuda.empty_cache()
    wl = WORKLOADS["si1728"]
    ci = synth.cell_inputs(wl["species"], wl["n"], 0)
    t0 = time.perf_counter()
    cell = pw.Cell(ci["L"], ci["tau"], ci["depth"], ci["dkb"], wl["ecut"], precision="mixed")
    pw.pw_cell_set_projectors(cell.h, True)
    tune = None
    if not args.no_autotune:
        fr = pw.pw_cell_autotune_fft(cell.h, 256, precision="mixed")
        tune = {"L": fr.best.L, "R": fr.best.R, "compact": fr.best.compact, "batch_mib": fr.best.batch_bytes >> 20,
                "ms_best_256_bands": fr.ms_best, "ms_default": fr.ms_default}
    nb = wl["nb"]
    s = pw.pw_solver_create(cell.h, nb, tol=0.0, seed=0, precision="mixed")
    t_setup = time.perf_counter() - t0
    try:
        w = pw.pw_subspace_step(cell.h, s)
        stream = torch.cuda.current_stream()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = pw.pw_subspace_step(cell.h, s)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        eig, _ = pw.pw_solver_eigs(s, nb)
    finally:
        pw.pw_solver_destroy(s)
        cell.close()
    return {"workload": wl["name"], "npw": cell.npw, "grid": list(cell.grid), "nbands": nb,
            "nproj": cell.nproj, "projectors": "generated on the fly", "nsub": r.nsub,
            "ms_per_step": ms, "iters_per_s": 1e3 / ms, "warmup_step_ms": w.ms, "warmup_nsub": w.nsub,
            "setup_s": t_setup, "finite": bool(np.isfinite(eig).all()),
            "stage_ms": {k: getattr(r, "ms_" + k) for k in ["resid", "hpsi", "gram", "rr", "rot"]},
            "rr_ms": {nm: r.ms_rr_part[i] for i, nm in
                      enumerate(["chol_inv", "transform", "tridiag", "dc", "backtransform"])},
            "autotune_fft": tune}


# ------------------------------------------------------------------ helpers --

def reduce_timing(ms: float, steps: int, world: int, device=None):
    """Replicas only: the slowest rank's time sets the job time; the value is
    the steps all ranks completed divided by it.  Returns (max_ms, iters/s)."""
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, world * steps / (ms / 1e3)

def step_flops(npw, nb, ns, k, nproj, grid, hcols=None):
    """Algorithmic FLOPs of one step (complex products counted as 8 real flops);
    hcols: columns H is applied to (k, or nb + 2k when H X and H P are fresh)."""
    import math
    hcols = k if hcols is None else hcols
    n3 = grid[0] * grid[1] * grid[2]
    fft = 2 * 5.0 * n3 * math.log2(n3) * hcols      # one inverse + one forward 3-D FFT per column
    proj = 2 * 8.0 * npw * nproj * hcols            # beta^H W and beta (D B)
    gram = 2 * 4.0 * npw * ns * ns                  # S^H S and S^H (H S), Hermitian halves
    # P' = [W P] C_WP and H P' (ns - nb), then X' = X C_X + P' and H X' (nb)
    rot = 2 * 8.0 * npw * nb * (ns - nb) + 2 * 8.0 * npw * nb * nb
    return dict(fft=fft, proj=proj, gram=gram, rot=rot, npw=npw)


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def hemv_slice_bytes(n):
    """Digit-slice bytes the tensor-core Hermitian products of the Householder
    reduction stream: each column c of a panel (32 columns from j0) whose
    trailing order n - j0 - 1 is at least HS_MIN_ORDER reads every lower
    trailing tile (128 x 128, real and imaginary parts, eight FP16 slices:
    512 KB) from tile (c + 1) // 128 on."""
    nt = (n + 127) // 128
    total = 0
    for j0 in range(0, n - 1, 32):
        if n - j0 - 1 < HS_MIN_ORDER:
            break
        for c in range(j0, min(j0 + 32, n - 1)):
            ntp = nt - (c + 1) // 128
            total += ntp * (ntp + 1) // 2 * 512 * 1024
    return total


def roofline(stage, rr_part, fl, n, nb, precision, fft=None):
    """Roofline of the dominant kernel, timed by the solver's CUDA events,
    plus the per-stage figures.

    Mixed precision: the dominant kernel is the split-FP16 tcgen05 GEMM
    (k_tc_gemm: S^H S, S M, H S M, S~^H H S~ and the rotations); it counts the
    tensor flops it issues (three slice products per real multiply-add) over
    its three stages' time against the measured sustained 16-bit rate.  The
    Householder stage counts the digit-slice bytes its tensor-core Hermitian
    products stream against the measured HBM copy rate (its time also holds
    the per-column FP64 kernels, the slicing and the panel updates).  The FFT
    stage counts its algorithmic c64 bytes against the HBM rate and its flops
    against the nominal FP32 rate.
    """
    mixed = precision == "mixed"
    parts = {k: v for k, v in stage.items() if k != "rr"}
    parts.update(rr_part)
    peaks = measured_peaks()
    tc_peak = peaks.get("bf16_tflops_sustained")
    hbm = peaks.get("hbm_gbs")
    tc_stages = [k for k in ("gram", "transform", "rot") if parts.get(k)]
    if mixed and tc_peak and tc_stages:
        t_ms = sum(parts[k] for k in tc_stages)
        tfl = sum(3 * tc_flops(k, fl, n, nb) for k in tc_stages)
        ach = tfl / (t_ms * 1e-3) / 1e12
        roof = {"bound": "tensor", "kernel": "k_tc_gemm (split-FP16 tcgen05 GEMM: S^H S; S M, H S M, "
                                              "S~^H H S~; rotations)",
                "stage": "tc_gemm", "ms": t_ms, "achieved": ach, "peak": tc_peak, "unit": "TFLOP/s",
                "frac": ach / tc_peak, "traffic": None, "algorithmic_flops": tfl,
                "peak_source": "of measured: bf16 sustained (fp16 has the same nominal rate)"}
    else:
        dom = max(parts, key=parts.get)
        roof = {"bound": None, "kernel": dom, "stage": dom, "ms": parts[dom]}
    # per-stage figures
    st = {}
    if mixed and tc_peak:
        for k in tc_stages:
            tfl = 3 * tc_flops(k, fl, n, nb)
            a = tfl / (parts[k] * 1e-3) / 1e12
            st["tc_gemm_" + k] = {"ms": parts[k], "tensor_tflops": a, "peak": tc_peak, "frac": a / tc_peak,
                                  "unit": "TFLOP/s (split-FP16 slice products, of measured sustained)"}
    if fft and hbm:
        a = fft["bytes"] / (fft["ms"] * 1e-3) / 1e9
        f = fft["flops"] / (fft["ms"] * 1e-3) / 1e12
        st["fft"] = {"ms": fft["ms"], "bands": fft["bands"], "achieved_gbs": a, "hbm_peak_gbs": hbm,
                     "frac_hbm": a / hbm, "tflops": f, "fp32_peak_tflops": FP32_PEAK_TFLOPS,
                     "frac_fp32": f / FP32_PEAK_TFLOPS, "bytes": fft["bytes"], "source": fft["source"]}
    if parts.get("tridiag") and hbm:
        sb = hemv_slice_bytes(n)
        a = sb / (parts["tridiag"] * 1e-3) / 1e9
        st["householder"] = {"ms": parts["tridiag"], "hemv_slice_bytes": sb, "achieved_gbs": a,
                             "hbm_peak_gbs": hbm, "frac_hbm": a / hbm,
                             "note": "slice bytes of the tensor-core Hermitian products over the whole "
                                     "reduction's time (which also holds k_pcol, k_prows, the slicing and "
                                     "the panel updates)"}
    roof["stages"] = st
    roof["stage_ms"] = stage
    roof["rr_ms"] = rr_part
    return roof


def tc_flops(stage, fl, n, nb):
    """Complex-product flops (8 per complex multiply-add) of a tensor-core stage
    of the mixed step: the Gram S^H S (Hermitian half), the transform
    S M, H S M (triangular M: half) and S~^H H S~ (Hermitian half), the
    rotations: with H blocks carried X' = S C, H X' = HS C, P' = S C_P and
    H P' = HS C_P (C_P's first nb rows zero: skipped), else P' = S C_P and
    X' = S~ Y."""
    npw = fl["npw"]
    if stage == "gram":
        return 4.0 * npw * n * n
    if stage == "transform":
        return 2 * 4.0 * npw * n * n + 4.0 * npw * n * n
    if stage == "rot":
        if fl.get("carried"):
            return 2 * (8.0 * npw * n * nb + 8.0 * npw * (n - nb) * nb)
        return 8.0 * npw * n * nb + 8.0 * npw * (n - nb) * nb
    return 0.0


class Clocks:
    """nvidia-smi samples during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None
        self.index = index

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
                for nm, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------ oracle sample --

def oracle_sample(wl, seed=0, frac_rows=32, apply_bands=8, rr_div=2):
    """One sampled oracle step: time its components on bounded pieces of the
    workload and scale them to a full step.  Returns (seconds_per_step, note,
    pieces) with pieces[name] = {measured_s, scale, scaled_s}."""
    import numpy as np
    import synth
    from oracle import pw_oracle as O
    ci = synth.cell_inputs(wl["species"], wl["n"], seed)
    if not hasattr(oracle_sample, "cell"):
        oracle_sample.cell = O.make_cell(ci["L"], ci["tau"], ci["depth"], ci["dkb"], wl["ecut"])
    cell = oracle_sample.cell
    nb, npw = wl["nb"], cell.npw
    ns = 3 * nb
    rng = np.random.default_rng(seed)
    t = {}

    def piece(name, sec, scale):
        t[name] = {"measured_s": sec, "scale": scale, "scaled_s": sec * scale}

    kb = min(apply_bands, nb)
    X = synth.draw_x0(seed, len(ci["tau"]), npw, kb)
    t0 = time.perf_counter()
    O.apply_H(cell, X)
    piece("hpsi", time.perf_counter() - t0, nb / kb)
    rows = max(ns, npw // frac_rows)
    S = rng.standard_normal((rows, ns)) + 1j * rng.standard_normal((rows, ns))
    t0 = time.perf_counter()
    S.conj().T @ S
    S.conj().T @ S
    piece("gram", time.perf_counter() - t0, npw / rows)
    C = rng.standard_normal((ns, nb)) + 1j * rng.standard_normal((ns, nb))
    t0 = time.perf_counter()
    for _ in range(2):
        S @ C
        S[:, nb:] @ C[nb:]
    piece("rot", time.perf_counter() - t0, npw / rows)
    m = ns // rr_div
    Ssm = rng.standard_normal((4 * m, m)) + 1j * rng.standard_normal((4 * m, m))
    Hs = rng.standard_normal((4 * m, 4 * m))
    Hs = Hs + Hs.T
    HSsm = Hs @ Ssm
    t0 = time.perf_counter()
    O.rayleigh_ritz(Ssm, HSsm, m // 3)
    # the Gram products inside rayleigh_ritz are at 4m rows; cubic part dominates
    piece("rr", time.perf_counter() - t0, rr_div ** 3)
    total = sum(v["scaled_s"] for v in t.values())
    note = (f"oracle components timed on bounded pieces and scaled to one full step: H on {kb} of "
            f"{nb} bands (x{nb // kb}); S^H S, S^H HS and the 4 rotations on {rows} of {npw} rows "
            f"(x{npw / rows:.1f}); Rayleigh-Ritz at order {m} of {ns} (x{rr_div ** 3}, cubic)")
    return total, note, t


def cpu_cores():
    try:
        from threadpoolctl import threadpool_info
        n = max((i.get("num_threads") or 0) for i in threadpool_info())
        if n:
            return int(n)
    except Exception:
        pass
    return os.cpu_count()


# ------------------------------------------------------------------- arms --

def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    wl = WORKLOADS[args.workload]
    for _ in range(args.warmup):
        oracle_sample(wl)
    secs, measured = [], []
    for _ in range(args.steps):
        s, note, parts = oracle_sample(wl)
        secs.append(s)
        measured.append(sum(p["measured_s"] for p in parts.values()))
    sec = sum(secs) / len(secs)
    v = 1.0 / sec
    cores = cpu_cores()
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "iters/s",
           "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": sec * 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": wl["name"], "nbands": wl["nb"], "precision": "fp64",
                      "implementation": "FP64 numpy/scipy oracle on host cores"},
           "cpu_baseline": {"value": v, "unit": "iters/s", "cores": cores, "kind": "oracle",
                            "sample": note, "extrapolated": True, "pieces": parts,
                            "measured_s_per_step": sum(measured) / len(measured)},
           "e2e": {"value": v, "unit": "iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_gpu(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import synth
    import paper_2406_10765_gb300 as pw

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    wl = WORKLOADS[args.workload]
    if args.workload == "si1728":
        # the largest cell: the step alone (FP64 comparison, full solves and the
        # extra Si-1728 object of the default line do not fit a short run)
        args.no_fp64 = args.no_e2e = args.no_accuracy = args.no_si1728 = True
    ci = synth.cell_inputs(wl["species"], wl["n"], 0)
    cell = pw.Cell(ci["L"], ci["tau"], ci["depth"], ci["dkb"], wl["ecut"], precision=args.precision)
    if wl.get("onthefly"):
        pw.pw_cell_set_projectors(cell.h, True)
    nb = wl["nb"]
    stream = torch.cuda.current_stream()
    tune = None
    if not args.no_autotune:
        # untimed set-up: the FFT plan of this cell, then per-shape K splits of
        # the tensor-core products on their first call (solver creation and
        # the first warm-up step)
        fr = pw.pw_cell_autotune_fft(cell.h, min(nb, 256), precision=args.precision)
        pw.pw_autotune_gemm(1)
        tune = {"fft": {"L": fr.best.L, "R": fr.best.R, "compact": fr.best.compact,
                        "batch_mib": fr.best.batch_bytes >> 20,
                        "ms_best": fr.ms_best, "ms_default": fr.ms_default,
                        "default": [fr.dflt.L, fr.dflt.R, fr.dflt.compact, fr.dflt.batch_bytes >> 20],
                        "candidates": fr.ncand, "bands": min(nb, 256),
                        "timed": [ln for ln in pw.pw_cell_fft_tune_log(cell.h).splitlines() if ln]}}
    solver = pw.pw_solver_create(cell.h, nb, tol=0.0, seed=0, precision=args.precision)
    for _ in range(args.warmup):
        pw.pw_subspace_step(cell.h, solver)

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    clocks = Clocks(local)
    barrier()
    clocks.start()
    launches0 = pw.pw_kernel_launches()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    reps = [pw.pw_subspace_step(cell.h, solver) for _ in range(args.steps)]
    e1.record(stream)
    barrier()
    launches = pw.pw_kernel_launches() - launches0
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    ms, value = reduce_timing(ms, args.steps, world, device="cuda")

    # roofline of the dominant stage, from the solver's CUDA events
    stage = {k: sum(getattr(r, "ms_" + k) for r in reps) / len(reps)
             for k in ["resid", "hpsi", "gram", "rr", "rot"]}
    rr_part = {nm: sum(r.ms_rr_part[i] for r in reps) / len(reps)
               for i, nm in enumerate(["chol_inv", "transform", "tridiag", "dc", "backtransform"])}
    ns = reps[-1].nsub
    k_act = reps[-1].nactive
    fl = step_flops(cell.npw, nb, ns, k_act, cell.nproj, cell.grid, reps[-1].hpsi_cols)
    # mixed: H applied only to W means H X and H P were carried (4 rotation products)
    fl["carried"] = args.precision == "mixed" and reps[-1].hpsi_cols == k_act
    fft = None
    if tune is not None:
        # the local part of H psi (FFT kernels, V multiply, kinetic), timed by
        # the autotuner with CUDA events on `bands` bands with the chosen plan
        import math
        N = cell.grid[0]
        ncol = len({(int(a), int(b)) for a, b, _ in cell.m})
        bands = tune["fft"]["bands"]
        zb = ncol * N * 8                                   # FP32 z-pencils of one band
        bpb = max(1, min(bands, (tune["fft"]["batch_mib"] << 20) // zb))
        n3 = cell.grid[0] * cell.grid[1] * cell.grid[2]
        per_band = 32.0 * cell.npw + 4.0 * zb + 4.0 * n3 / bpb
        fft = {"ms": tune["fft"]["ms_best"], "bands": bands, "bytes": per_band * bands,
               "flops": 2 * 5.0 * n3 * math.log2(n3) * bands,
               "source": f"autotuner CUDA events, {bands} bands; bytes per band 32 npw (c128 sphere in and "
                         f"out) + 4 x 8 Ncol N (c64 z-pencils, Ncol {ncol}) + 4 N^3 / {bpb} (FP32 V per batch)"}
    roof = roofline(stage, rr_part, fl, ns, nb, args.precision, fft)
    roof["hpsi_cols"] = reps[-1].hpsi_cols
    out = {"metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f64" if args.precision == "fp64" else "f16x2-split tensor + f32 FFT + f64 dense",
           "data": "synthetic",
           "config": {"workload": wl["name"], "npw": cell.npw, "grid": list(cell.grid),
                      "nbands": nb, "nproj": cell.nproj, "nsub": ns, "precision": args.precision,
                      "l2": "inputs larger than L2 (S blocks of several GB)",
                      "parallelism": f"replicas x{world}"},
           "roofline": roof, "gpu_launches": launches, "launches_before_timed": launches0,
           "clocks": clk}
    if tune is not None:
        lines = [ln for ln in pw.pw_autotune_gemm_table().splitlines() if ln]
        tune["gemm_shapes_tuned"] = len(lines)
        tune["gemm_split_gt1"] = [ln for ln in lines if "split=1 " not in ln]
        out["config"]["autotune"] = tune
    pw.pw_solver_destroy(solver)

    if args.precision == "mixed" and not args.no_fp64:
        # the same step in FP64 (one warm-up, one timed): the "mixed vs FP64" ratio
        cell.set_precision("fp64")
        s64 = pw.pw_solver_create(cell.h, nb, tol=0.0, seed=0, precision="fp64")
        pw.pw_subspace_step(cell.h, s64)
        barrier()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        pw.pw_subspace_step(cell.h, s64)
        f1.record(stream)
        barrier()
        ms64 = f0.elapsed_time(f1)
        pw.pw_solver_destroy(s64)
        cell.set_precision("mixed")
        out["fp64_comparison"] = {"iters_per_s": 1e3 / ms64, "ms_per_step": ms64,
                                  "mixed_speedup": ms64 / (ms / args.steps)}

    x0h = torch.empty((nb, cell.npw), dtype=torch.complex128).pin_memory()
    x0h.copy_(torch.from_numpy(np.ascontiguousarray(synth.draw_x0(0, len(ci["tau"]), cell.npw, nb).T)))
    x0 = x0h.numpy().T          # Fortran-ordered view of the pinned buffer
    if not args.no_e2e:
        # the step rate end to end through pw_eigsolve with host buffers: the
        # pinned host start block in, H X0 and the initial Rayleigh-Ritz,
        # e2e_steps full steps (tol 0: no band locks, the timed step's work),
        # the FP64 polish, eigenvalues back to the host
        barrier()
        t0 = time.perf_counter()
        eig, rep, st = pw.pw_eigsolve(cell.h, nb, tol=0.0, maxit=args.e2e_steps, x0=x0,
                                      precision=args.precision, raise_noconv=False)
        barrier()
        t1 = time.perf_counter() - t0
        out["e2e"] = {"value": rep.iters / t1, "unit": "iters/s",
                      "h2d_bytes_per_step": x0.nbytes // max(1, rep.iters),
                      "d2h_bytes_per_step": eig.nbytes // max(1, rep.iters),
                      "iters": rep.iters, "seconds": t1, "status": int(st),
                      "note": f"pw_eigsolve (tol 0, {args.e2e_steps} full steps) from a pinned host start "
                              "block: upload, H X0, initial Rayleigh-Ritz, the steps, FP64 polish, "
                              "eigenvalues back to the host"}

    def section(key, fn):
        # a rank-0 part of the line after the timed steps: a failure is
        # recorded under its key instead of losing the measured line
        try:
            out[key] = fn()
        except Exception as exc:
            out[key] = {"error": f"{type(exc).__name__}: {exc}"}

    def cpu_baseline():
        sec, note, parts = oracle_sample(wl)
        return {"value": 1.0 / sec, "unit": "iters/s", "cores": cpu_cores(),
                "kind": "oracle", "sample": note, "extrapolated": True, "pieces": parts,
                "measured_s_per_step": sum(p["measured_s"] for p in parts.values())}

    if rank == 0 and not args.no_accuracy and args.precision == "mixed":
        section("accuracy", lambda: accuracy_run(pw, torch, cell, nb, x0, torch.cuda.synchronize))
    if rank == 0 and not args.no_serve:
        section("serving", lambda: serve_sweep(args))
    if rank == 0 and not args.no_si1728 and args.precision == "mixed":
        cell.close()
        section("si1728", lambda: si1728_step(pw, torch, args))
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        section("cpu_baseline", cpu_baseline)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_serve_only(args):
    import torch
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    sv = serve_sweep(args)
    last = sv["rates"][-1]
    print(json.dumps({"metric": "served fixed-potential eigensolves (solves/s)", "value": last["solves_per_s"],
                      "unit": "solves/s", "n_gpus": 1, "higher_is_better": True, "data": "synthetic",
                      "config": {"workload": "seeded serving stream (Si/C, n 1..3, Ecut 8-12 Ha)"},
                      "serving": sv}), flush=True)


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    elif a.serve_only:
        run_serve_only(a)
    else:
        run_gpu(a)
