"""Small, self-contained cases of the hot kernels for profiler captures.

    python -m paper_2406_10765_gb300.profile_cases <case> [--reps N]

Cases (each holds at most a few GB on the device and runs its kernels a few
times after one warm-up):
  step64      one FP64 LOBPCG step on the Si 64-atom cell (2x2x2, Ecut 10 Ha,
              npw 13,056, 144 bands): k_zgemm, FFT kernels, Rayleigh-Ritz
  step64mix   the same step in mixed precision (k_tc_gemm)
  step512mix  one mixed-precision LOBPCG step on the Si 512-atom cell (the
              bench workload; solver creation included)
  tcgemm      split-FP16 tensor-core A^H A, A: 104,415 x 1,152 complex
  smgemm      split-FP16 tensor-core S M, S: 30,000 x 3,456, M: 3,456 x 3,456
              complex (the shape class of the Rayleigh-Ritz transform S M)
  heev        FP64 Hermitian eigensolver, n = 1,152 (Householder, D&C);
              --n 3456 gives the Si-512 Rayleigh-Ritz order
  ozgemm      FP64-accurate tensor-core product C = M Y of the Rayleigh-Ritz
              finish at Si-512 (M 3,456 x 3,456 upper triangular, Y 3,456 x
              1,152 complex), against numpy in FP64
  hpsi512     FP64 H psi on 16 bands of the Si 512-atom cell (grid 96^3)
  hpsi512mix  mixed-precision H psi on --nb bands (default 1152) of the same cell
  projmodes   H psi of the Si-512 cell with resident and with on-the-fly
              projectors: mixed on 1,152 bands, FP64 on 64 (CUDA-event times)
  step1728mix the 1,728-atom cell (Ecut 8 Ha, grid 128^3, npw 251,967, 6,912
              projectors generated on the fly), 3,840 bands in mixed
              precision: solver creation and --reps LOBPCG steps with stage
              times, device memory in use, and the Rayleigh-Ritz property
              that no Ritz value rises.  Holds ~250 GB: not a profiler case.
"""
from __future__ import annotations

import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("case")
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--n", type=int, default=1152, help="order of the heev case")
    ap.add_argument("--nb", type=int, default=1152, help="bands of the hpsi512mix case")
    a = ap.parse_args()
    import numpy as np
    import torch

    import synth
    import paper_2406_10765_gb300 as pw

    torch.cuda.set_device(0)
    if a.case in ("step64", "step64mix", "step512mix"):
        prec = "fp64" if a.case == "step64" else "mixed"
        ncell, nbands = (4, 1152) if a.case == "step512mix" else (2, 144)
        ci = synth.cell_inputs("Si", ncell, 0)
        cell = pw.Cell(ci["L"], ci["tau"], ci["depth"], ci["dkb"], 10.0, precision=prec)
        s = pw.pw_solver_create(cell.h, nbands, tol=0.0, seed=0, precision=prec)
        l0 = pw.pw_kernel_launches()
        r = pw.pw_subspace_step(cell.h, s)
        l1 = pw.pw_kernel_launches()
        for _ in range(a.reps):
            l0 = pw.pw_kernel_launches()
            r = pw.pw_subspace_step(cell.h, s)
            l1 = pw.pw_kernel_launches()
        print(f"{a.case}: npw {cell.npw}, last step {r.ms:.1f} ms, launches before it {l0}, "
              f"in it {l1 - l0}")
        pw.pw_solver_destroy(s)
    elif a.case == "step1728mix":
        import time
        ci = synth.cell_inputs("Si", 6, 0)
        cell = pw.Cell(ci["L"], ci["tau"], ci["depth"], ci["dkb"], 8.0, precision="mixed")
        pw.pw_cell_set_projectors(cell.h, True)
        nb = 3840
        t0 = time.time()
        s = pw.pw_solver_create(cell.h, nb, tol=0.0, seed=0, precision="mixed")
        free, total = torch.cuda.mem_get_info()
        e0, r0 = pw.pw_solver_eigs(s, nb)
        print(f"step1728mix: npw {cell.npw}, grid {cell.grid}, create {time.time() - t0:.1f} s, "
              f"device in use {(total - free) / 2**30:.1f} GiB of {total / 2**30:.1f}")
        print(f"  start: theta [{e0[0]:.6f}, {e0[-1]:.6f}], max resid {r0.max():.3e}")
        for it in range(max(1, a.reps)):
            r = pw.pw_subspace_step(cell.h, s)
            e1, r1 = pw.pw_solver_eigs(s, nb)
            print(f"  step {it + 1}: {r.ms:.0f} ms (resid {r.ms_resid:.0f}, hpsi {r.ms_hpsi:.0f} on "
                  f"{r.hpsi_cols} cols, gram {r.ms_gram:.0f}, rr {r.ms_rr:.0f} "
                  f"[{', '.join(f'{v:.0f}' for v in r.ms_rr_part)}], rot {r.ms_rot:.0f}), nsub {r.nsub}")
            print(f"    theta [{e1[0]:.6f}, {e1[-1]:.6f}], max rise {np.max(e1 - e0):.3e}, "
                  f"max resid {r1.max():.3e}, finite {bool(np.isfinite(e1).all())}")
            e0 = e1
        pw.pw_solver_destroy(s)
    elif a.case == "tcgemm":
        k, m = 104415, 1152
        A = (torch.randn(m, k, dtype=torch.complex128, device="cuda") / k ** 0.5).T
        for _ in range(a.reps + 1):
            C = pw.pw_zgemm_tc("C", A, A)
        torch.cuda.synchronize()
        print("tcgemm done", float(C.abs().max()))
    elif a.case == "smgemm":
        g = torch.Generator(device="cuda").manual_seed(0)
        npw, n = 30000, 3456
        S = (torch.randn(n, npw, dtype=torch.complex128, device="cuda", generator=g) * 1e-2).T
        M = torch.randn(n, n, dtype=torch.complex128, device="cuda", generator=g).T
        for _ in range(a.reps + 1):
            C = pw.pw_zgemm_tc("N", S, M)
        torch.cuda.synchronize()
        print("smgemm done", float(C.abs().max()))
    elif a.case == "ozgemm":
        n, nb = 3456, 1152
        rng = np.random.default_rng(0)
        M = np.triu(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
        Y = rng.standard_normal((n, nb)) + 1j * rng.standard_normal((n, nb))
        Md = torch.from_numpy(np.asfortranarray(M)).cuda().T.contiguous().T
        Yd = torch.from_numpy(np.asfortranarray(Y)).cuda().T.contiguous().T
        for _ in range(1 + a.reps):
            C = pw.pw_zgemm_f64tc("N", "N", Md, Yd)
        torch.cuda.synchronize()
        ref = M @ Y
        err = np.abs(C.cpu().numpy() - ref).max() / np.abs(ref).max()
        print(f"ozgemm: {n} x {nb} x {n}, max error / max |C| {err:.2e}")
    elif a.case == "heev":
        n = a.n
        rng = np.random.default_rng(0)
        M = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
        H = torch.from_numpy(M + M.conj().T).cuda()
        for _ in range(a.reps + 1):
            w, Y = pw.pw_heev(H, n // 3)
        torch.cuda.synchronize()
        print("heev done", float(w[0]))
    elif a.case == "hpsi512":
        ci = synth.cell_inputs("Si", 4, 0)
        cell = pw.Cell(ci["L"], ci["tau"], ci["depth"], ci["dkb"], 10.0)
        x = pw.new_block(cell.npw, 16)
        x.copy_(torch.from_numpy(synth.draw_x0(0, 512, cell.npw, 16)))
        y = pw.new_block(cell.npw, 16)
        for _ in range(a.reps + 1):
            pw.pw_apply_H(cell.h, x, y)
        torch.cuda.synchronize()
        print("hpsi512 done")
    elif a.case == "hpsi512mix":
        ci = synth.cell_inputs("Si", 4, 0)
        cell = pw.Cell(ci["L"], ci["tau"], ci["depth"], ci["dkb"], 10.0, precision="mixed")
        x = pw.new_block(cell.npw, a.nb)
        x.copy_(torch.from_numpy(synth.draw_x0(0, 512, cell.npw, a.nb)))
        y = pw.new_block(cell.npw, a.nb)
        for _ in range(a.reps + 1):
            pw.pw_apply_H(cell.h, x, y)
        torch.cuda.synchronize()
        print("hpsi512mix done")
    elif a.case == "projmodes":
        ci = synth.cell_inputs("Si", 4, 0)
        for prec, nb in (("mixed", 1152), ("fp64", 64)):
            cell = pw.Cell(ci["L"], ci["tau"], ci["depth"], ci["dkb"], 10.0, precision=prec)
            x = pw.new_block(cell.npw, nb)
            x.copy_(torch.from_numpy(synth.draw_x0(0, 512, cell.npw, nb)))
            y = pw.new_block(cell.npw, nb)
            for mode in (False, True):
                pw.pw_cell_set_projectors(cell.h, mode)
                pw.pw_apply_H(cell.h, x, y)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                for _ in range(a.reps):
                    pw.pw_apply_H(cell.h, x, y)
                e1.record()
                torch.cuda.synchronize()
                print(f"projmodes {prec} nb={nb} {'on-the-fly' if mode else 'resident'}: "
                      f"{e0.elapsed_time(e1) / a.reps:.1f} ms per H psi")
            cell.close()
    else:
        raise SystemExit(f"unknown case {a.case}")


if __name__ == "__main__":
    main()
