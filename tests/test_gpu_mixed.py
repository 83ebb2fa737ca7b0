"""Mixed-precision path (FP32 FFTs, split-FP16 tensor-core contractions, FP64
Cholesky / eigensolve / residual norms) against the FP64 oracle at the stated
tolerances: |d eps| <= 1e-6 Ha, residual <= 1e-5, ||X^H X - I|| <= 1e-10."""
import os

import numpy as np
import pytest

import synth
from oracle import pw_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from gpu_util import cells, to_dev, rel  # noqa: E402

GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("species,ecut,nb,gold", [("Si", 10.0, 24, "si8_ecut10_seed0_eigs.txt"),
                                                  ("C", 8.0, 18, "c8_ecut8_seed0_eigs.txt")])
def test_mixed_eigsolve_tolerances(species, ecut, nb, gold):
    import paper_2406_10765_gb300 as pw
    lib, orc, _ = cells(species, 1, ecut)
    ref = np.loadtxt(os.path.join(GOLD, gold))[:nb]
    psi = pw.new_block(lib.npw, nb)
    # the split-precision residual floor is ~1e-6; the stated targets are
    # |d eps| <= 1e-6 Ha, residual <= 1e-5, ||X^H X - I|| <= 1e-10
    eig, rep, st = pw.pw_eigsolve(lib.h, nb, tol=5e-6, maxit=300, seed=0, precision="mixed",
                                  psi_out=psi)
    assert np.abs(eig - ref).max() <= 1e-6
    assert rep.max_resid <= 1e-5
    assert rep.orth_err <= 1e-10
    # residual recomputed by the oracle from the returned block
    X = psi.cpu().numpy()
    R = O.apply_H(orc, X) - X * eig[None, :]
    assert np.sqrt((np.abs(R) ** 2).sum(axis=0)).max() <= 1e-5


def test_mixed_step_tracks_fp64_step():
    import paper_2406_10765_gb300 as pw
    lib, orc, _ = cells("Si", 1, 10.0)
    nb = 24
    x0 = synth.draw_x0(0, 8, orc.npw, nb)
    a = pw.pw_solver_create(lib.h, nb, tol=0.0, x0=x0, precision="fp64")
    b = pw.pw_solver_create(lib.h, nb, tol=0.0, x0=x0, precision="mixed")
    for _ in range(3):
        pw.pw_subspace_step(lib.h, a)
        pw.pw_subspace_step(lib.h, b)
    ea, _ = pw.pw_solver_eigs(a, nb)
    eb, _ = pw.pw_solver_eigs(b, nb)
    assert np.abs(ea - eb).max() < 1e-4
    pw.pw_solver_destroy(a)
    pw.pw_solver_destroy(b)


def test_mixed_apply_h_si512_sampled():
    lib, orc, _ = cells("Si", 4, 10.0, precision="mixed")
    import paper_2406_10765_gb300 as pw
    nb = 24
    x = synth.draw_x0(1, 512, orc.npw, nb)
    out = pw.new_block(lib.npw, nb)
    pw.pw_apply_H(lib.h, to_dev(x), out)
    got = out.cpu().numpy()
    for j in [0, 23]:
        ref = O.apply_H(orc, x[:, j:j + 1])[:, 0]
        assert rel(got[:, j], ref) < 1e-5


def test_mixed_steps_track_oracle_si64():
    # mixed precision on the 64-atom cell (Rayleigh-Ritz order 432; the
    # tensor-core products span many 128 x 128 tiles with ragged edges):
    # the Ritz values stay within the split-precision error of the oracle's
    # FP64 steps from the same start block
    import paper_2406_10765_gb300 as pw
    lib, orc, _ = cells("Si", 2, 10.0, precision="mixed")
    nb = 144
    x0 = synth.draw_x0(0, 64, orc.npw, nb)
    st = O.lobpcg_init(orc, x0)
    s = pw.pw_solver_create(lib.h, nb, tol=0.0, x0=x0, precision="mixed")
    for _ in range(3):
        st = O.lobpcg_step(orc, st)
        pw.pw_subspace_step(lib.h, s)
    e, _ = pw.pw_solver_eigs(s, nb)
    assert np.abs(e - st.lam).max() < 1e-4
    pw.pw_solver_destroy(s)


def test_mixed_chunked_tall_products_si64():
    # the tall split-FP16 products (Gram, S M, A~, rotations) taken over
    # plane-wave chunks of 1,000 rows (a ragged last chunk) follow the
    # single-chunk solver and the oracle's FP64 steps
    import paper_2406_10765_gb300 as pw
    lib, orc, _ = cells("Si", 2, 10.0, precision="mixed")
    nb = 144
    x0 = synth.draw_x0(0, 64, orc.npw, nb)
    assert orc.npw % 1000 != 0 and orc.npw > 5000
    st = O.lobpcg_init(orc, x0)
    a = pw.pw_solver_create(lib.h, nb, tol=0.0, x0=x0, precision="mixed")
    b = pw.pw_solver_create(lib.h, nb, tol=0.0, x0=x0, precision="mixed", chunk_rows=1000)
    for _ in range(3):
        st = O.lobpcg_step(orc, st)
        pw.pw_subspace_step(lib.h, a)
        pw.pw_subspace_step(lib.h, b)
    ea, _ = pw.pw_solver_eigs(a, nb)
    eb, rb = pw.pw_solver_eigs(b, nb)
    assert np.abs(eb - ea).max() < 1e-6
    assert np.abs(eb - st.lam).max() < 1e-4
    assert np.isfinite(rb).all()
    pw.pw_solver_destroy(a)
    pw.pw_solver_destroy(b)


def test_mixed_chunked_eigsolve_si8():
    # a full mixed solve with chunks of 250 plane-wave rows meets the same
    # targets against the stored FP64 eigenvalues
    import paper_2406_10765_gb300 as pw
    lib, orc, _ = cells("Si", 1, 10.0)
    nb = 24
    ref = np.loadtxt(os.path.join(GOLD, "si8_ecut10_seed0_eigs.txt"))[:nb]
    eig, rep, st = pw.pw_eigsolve(lib.h, nb, tol=5e-6, maxit=300, seed=0, precision="mixed",
                                  chunk_rows=250)
    assert np.abs(eig - ref).max() <= 1e-6
    assert rep.max_resid <= 1e-5
    assert rep.orth_err <= 1e-10


def test_mixed_steps_with_k_split():
    # every tensor-core product of the step with its K range cut in three
    # (including the triangular and zero-block K bounds of S M and P') tracks
    # the oracle's FP64 steps as the single-part products do
    import paper_2406_10765_gb300 as pw
    lib, orc, _ = cells("Si", 2, 10.0, precision="mixed")
    nb = 144
    x0 = synth.draw_x0(0, 64, orc.npw, nb)
    st = O.lobpcg_init(orc, x0)
    try:
        pw.pw_autotune_gemm(2, 3)
        s = pw.pw_solver_create(lib.h, nb, tol=0.0, x0=x0, precision="mixed")
        for _ in range(3):
            st = O.lobpcg_step(orc, st)
            pw.pw_subspace_step(lib.h, s)
        e, _ = pw.pw_solver_eigs(s, nb)
        pw.pw_solver_destroy(s)
    finally:
        pw.pw_autotune_gemm(0)
    assert np.abs(e - st.lam).max() < 1e-4


def test_mixed_steps_si512_full_size_sampled():
    # the timed configuration of the benchmark (Si-512, 1,152 bands, mixed,
    # steps with nsub 2,304 then 3,456): no Ritz value rises; on sampled bands
    # the Rayleigh quotient and residual norm of the returned vectors under
    # the oracle's FP64 operator equal the solver's Ritz values and residual
    # norms, and the sampled block is orthonormal
    import paper_2406_10765_gb300 as pw
    lib, orc, _ = cells("Si", 4, 10.0, precision="mixed")
    nb = 1152
    s = pw.pw_solver_create(lib.h, nb, tol=0.0, seed=0, precision="mixed")
    e_prev, _ = pw.pw_solver_eigs(s, nb)
    nsubs = []
    for _ in range(2):
        rep = pw.pw_subspace_step(lib.h, s)
        nsubs.append(rep.nsub)
        e, resid = pw.pw_solver_eigs(s, nb)
        assert np.all(e <= e_prev + 1e-9)
        e_prev = e
    assert nsubs == [2 * nb, 3 * nb]
    X = pw.new_block(lib.npw, nb)
    pw.pw_solver_block(s, X)
    pw.pw_solver_destroy(s)
    cols = [0, 1, 575, nb - 1]
    xs = X[:, cols].cpu().numpy()
    hx = O.apply_H(orc, xs)
    for k, j in enumerate(cols):
        x, h = xs[:, k], hx[:, k]
        rho = np.vdot(x, h).real / np.vdot(x, x).real
        assert abs(rho - e[j]) < 1e-5, (j, rho, e[j])
        r = np.linalg.norm(h - e[j] * x)
        assert abs(r - resid[j]) < 1e-5 * max(1.0, r), (j, r, resid[j])
    g = xs.conj().T @ xs
    assert np.abs(g - np.eye(len(cols))).max() < 1e-5


def test_mixed_h_blocks_carried_then_fresh_si64():
    # H X and H P carried through the split-precision rotations hold the
    # split products' error: carried all the way (h_blocks 2) the residual
    # stalls near 1e-4 and the eigenvalues stay far above 1e-6 Ha off; carried
    # only while the residual is above 1e-3 and applied afresh after that (1)
    # the solve reaches 5e-6 and the FP64 eigenvalues to 1e-6 Ha, as applying
    # H to [X W P] every step (0, the default) does
    import paper_2406_10765_gb300 as pw
    lib, orc, _ = cells("Si", 2, 10.0, precision="mixed")
    nb = 144
    x0 = synth.draw_x0(0, 64, orc.npw, nb)
    ref, _, _ = pw.pw_eigsolve(lib.h, nb, tol=1e-9, maxit=400, x0=x0, precision="fp64")
    s = pw.pw_solver_create(lib.h, nb, tol=0.0, x0=x0, precision="mixed", h_blocks=2)
    floor = np.inf
    for _ in range(100):
        pw.pw_subspace_step(lib.h, s)
        e, r = pw.pw_solver_eigs(s, nb)
        floor = min(floor, r.max())
    pw.pw_solver_destroy(s)
    assert floor > 3e-5
    assert np.abs(e - ref).max() > 1e-6
    for hb in (0, 1):
        e, rep, st = pw.pw_eigsolve(lib.h, nb, tol=5e-6, maxit=400, x0=x0, precision="mixed", h_blocks=hb)
        assert st == 0 and rep.max_resid <= 5e-6
        assert np.abs(e - ref).max() <= 1e-6


def test_mixed_step_reports_h_columns():
    # far from convergence mode 1 applies H once per step, to W; the default
    # applies it to X, W and P
    import paper_2406_10765_gb300 as pw
    lib, orc, _ = cells("Si", 1, 10.0, precision="mixed")
    nb = 24
    s = pw.pw_solver_create(lib.h, nb, tol=0.0, seed=1, precision="mixed", h_blocks=1)
    rep = pw.pw_subspace_step(lib.h, s)
    rep = pw.pw_subspace_step(lib.h, s)
    assert rep.max_resid > 1e-3 and rep.hpsi_cols == rep.nactive
    pw.pw_solver_destroy(s)
    s = pw.pw_solver_create(lib.h, nb, tol=0.0, seed=1, precision="mixed")
    pw.pw_subspace_step(lib.h, s)
    rep = pw.pw_subspace_step(lib.h, s)
    assert rep.hpsi_cols == nb + 2 * rep.nactive
    pw.pw_solver_destroy(s)
