"""The 1,728-atom cell (6x6x6 diamond cells, Ecut 8 Ha, npw 251,967, grid
128^3, 3,840 bands, 6,912 projectors generated on the fly) through two mixed
LOBPCG steps -- the Rayleigh-Ritz orders 7,680 and 11,520 on one GPU -- with
the step-level checks of the Si-512 test: no Ritz value rises, and on sampled
bands the Rayleigh quotient and residual norm under the oracle's FP64
operator equal the solver's values."""
import gc

import numpy as np
import pytest

import synth
from oracle import pw_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _oracle_h(ci, m, x):
    # the oracle's operator at this size, its projectors formed 64 atoms at a time
    Ls = np.full(3, float(ci["L"]) if np.ndim(ci["L"]) == 0 else ci["L"][0])
    Ns = (128, 128, 128)
    V = O.vloc_grid(Ls, Ns, ci["tau"], ci["depth"], 1.2)
    orc = O.Cell(Ls=Ls, Ns=Ns, ecut=8.0, m=m, kin=O.kinetic(m, Ls), V=V,
                 beta=np.zeros((m.shape[0], 0), complex), D=np.zeros(0))
    h = orc.kin[:, None] * x + O.apply_local(orc, x)
    D = np.asarray(ci["dkb"], float).reshape(-1)
    for a0 in range(0, len(ci["tau"]), 64):
        b = O.projectors(m, Ls, ci["tau"][a0:a0 + 64], 1.2)
        h += b @ (D[4 * a0:4 * a0 + b.shape[1], None] * (b.conj().T @ x))
    return h


def test_si1728_mixed_steps_sampled():
    import paper_2406_10765_gb300 as pw
    gc.collect()
    torch.cuda.empty_cache()
    ci = synth.cell_inputs("Si", 6, 0)
    lib = pw.Cell(ci["L"], ci["tau"], ci["depth"], ci["dkb"], 8.0, precision="mixed")
    assert lib.npw == 251967 and lib.grid == (128, 128, 128) and lib.nproj == 6912
    pw.pw_cell_set_projectors(lib.h, True)
    nb = 3840
    s = pw.pw_solver_create(lib.h, nb, tol=0.0, seed=0, precision="mixed")
    try:
        e_prev, _ = pw.pw_solver_eigs(s, nb)
        nsubs = []
        for _ in range(2):
            rep = pw.pw_subspace_step(lib.h, s)
            nsubs.append(rep.nsub)
            e, resid = pw.pw_solver_eigs(s, nb)
            assert np.all(np.isfinite(e)) and np.all(e <= e_prev + 1e-9)
            e_prev = e
        assert nsubs == [2 * nb, 3 * nb]
        cols = [0, 1, 1919, nb - 1]
        X = pw.new_block(lib.npw, nb)
        pw.pw_solver_block(s, X)
        xs = X[:, cols].cpu().numpy()
        del X
    finally:
        pw.pw_solver_destroy(s)
        lib.close()
        torch.cuda.empty_cache()
    Ls = np.full(3, float(ci["L"]) if np.ndim(ci["L"]) == 0 else ci["L"][0])
    m = O.sphere(8.0, Ls)
    hx = _oracle_h(ci, m, xs)
    for k, j in enumerate(cols):
        x, h = xs[:, k], hx[:, k]
        rho = np.vdot(x, h).real / np.vdot(x, x).real
        assert abs(rho - e[j]) < 1e-5, (j, rho, e[j])
        r = np.linalg.norm(h - e[j] * x)
        assert abs(r - resid[j]) < 1e-5 * max(1.0, r), (j, r, resid[j])
    g = xs.conj().T @ xs
    assert np.abs(g - np.eye(len(cols))).max() < 1e-5
