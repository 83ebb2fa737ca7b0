"""H psi on the GPU against the oracle (Sec. II-A Eq. 1 operator; FFT local
term of Sec. II-B, nonlocal term of Sec. III-A)."""
import numpy as np
import pytest

import synth
from oracle import pw_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from gpu_util import cells, to_dev, rel  # noqa: E402


def _run(lib, x, ld=None):
    import paper_2406_10765_gb300 as pw
    psi = to_dev(x, ld)
    npw, nb = x.shape
    if ld is None:
        out = pw.new_block(npw, nb)
    else:
        out = torch.zeros((nb, ld), dtype=torch.complex128, device="cuda").T
    pw.pw_apply_H(lib.h, psi, out)
    torch.cuda.synchronize()
    return out[:npw].cpu().numpy()


@pytest.mark.parametrize("species,n,ecut,nb", [("Si", 1, 10.0, 24), ("C", 1, 8.0, 37), ("Si", 1, 4.0, 5)])
def test_apply_h_fp64_matches_oracle(species, n, ecut, nb):
    lib, orc, _ = cells(species, n, ecut)
    assert lib.npw == orc.npw and np.array_equal(lib.m, orc.m) and lib.grid == orc.Ns
    x = synth.draw_x0(3, 8 * n ** 3, orc.npw, nb)
    got = _run(lib, x)
    assert rel(got, O.apply_H(orc, x)) < 1e-12


def test_apply_h_padded_ld_and_ragged_batch():
    lib, orc, _ = cells("Si", 1, 10.0)
    x = synth.draw_x0(4, 8, orc.npw, 83)       # more bands than one L2 batch? no: ragged tiles
    got = _run(lib, x, ld=orc.npw + 13)
    assert rel(got, O.apply_H(orc, x)) < 1e-12


def test_apply_h_orthorhombic_odd_grid():
    import paper_2406_10765_gb300 as pw
    Ls = np.array([9.0, 11.0, 7.5])
    tau = np.array([[0.5, 1.0, 2.0], [4.0, 6.0, 5.0], [8.0, 2.0, 1.0]])
    depth = np.array([-1.0, -0.95, -1.05])
    dkb = np.array([[0.7, 0.9, 1.1, 1.3], [0.6, 0.8, 1.0, 1.2], [1.4, 0.5, 0.9, 1.0]])
    grid = (18, 27, 16)
    lib = pw.Cell(Ls, tau, depth, dkb, 6.0, grid=grid)
    orc = O.make_cell(Ls, tau, depth, dkb, 6.0, grid=grid)
    assert lib.npw == orc.npw and np.array_equal(lib.m, orc.m)
    x = synth.draw_x0(5, 3, orc.npw, 7)
    assert rel(_run(lib, x), O.apply_H(orc, x)) < 1e-12


def test_apply_h_mixed_precision_error():
    lib, orc, _ = cells("Si", 1, 10.0, precision="mixed")
    x = synth.draw_x0(6, 8, orc.npw, 16)
    err = rel(_run(lib, x), O.apply_H(orc, x))
    assert err < 1e-5


def test_apply_h_si512_sampled_bands():
    # full-size cell (npw 104,415, grid 96^3) in the bench launch shape, with
    # a band block spanning several L2 batches; sampled bands vs the oracle
    lib, orc, ci = cells("Si", 4, 10.0)
    assert lib.npw == 104415 and lib.grid == (96, 96, 96)
    nb = 40
    x = synth.draw_x0(0, 512, orc.npw, nb)
    got = _run(lib, x)
    for j in [0, 17, 39]:
        ref = O.apply_H(orc, x[:, j:j + 1])[:, 0]
        assert rel(got[:, j], ref) < 1e-12


def test_supercell_folding_on_gpu():
    # eigenvector of the 8-atom cell folded into the 64-atom cell is an
    # eigenvector of the GPU operator with the same eigenvalue
    import paper_2406_10765_gb300 as pw
    small = synth.periodic_depths("Si", 1, 3)
    big = synth.periodic_depths("Si", 2, 3)
    cs = O.make_cell(small["L"], small["tau"], small["depth"], small["dkb"], 10.0)
    w, v = O.dense_eigs(cs, 4)
    lib = pw.Cell(big["L"], big["tau"], big["depth"], big["dkb"], 10.0)
    index = {tuple(mm): i for i, mm in enumerate(lib.m)}
    c = np.zeros((lib.npw, 4), complex)
    for i, mm in enumerate(cs.m):
        c[index[tuple(2 * mm)], :] = v[i, :]
    got = _run(lib, c)
    assert np.abs(got - c * w[None, :]).max() < 1e-12


def test_apply_h_argument_errors():
    import paper_2406_10765_gb300 as pw
    lib, orc, _ = cells("C", 1, 8.0)
    x = to_dev(synth.draw_x0(1, 8, orc.npw, 2))
    y = torch.empty_like(x)
    # nb = 0 is a no-op; ld < npw is rejected
    import ctypes as ct
    from paper_2406_10765_gb300 import binding as B
    st = B._stream(None)
    assert B._apply(lib.h, B._dptr(x), orc.npw, 0, B._dptr(y), st) == 0
    assert B._apply(lib.h, B._dptr(x), orc.npw - 1, 2, B._dptr(y), st) == B.PW_ERR_ARG
    assert B._apply(lib.h, ct.c_void_p(), orc.npw, 2, B._dptr(y), st) == B.PW_ERR_ARG


# every grid size with a register line-FFT kernel (and the Stockham fallback
# at 54 and 81): H psi on the Si 8-atom cell on an explicit grid against the
# oracle on the same grid; FP64 where the FP64 plane fits in shared memory
@pytest.mark.parametrize("N", [16, 24, 32, 36, 48, 54, 64, 72, 81, 96, 128, 144])
def test_apply_h_grid_sizes(N):
    ecut = 4.0 if N < 24 else 8.0
    x = None
    for prec, tol in (("fp64", 1e-12), ("mixed", 1e-5)):
        if prec == "fp64" and N * (N + 1) * 16 > 227 * 1024:
            continue
        lib, orc, _ = cells("Si", 1, ecut, grid=(N, N, N), precision=prec)
        assert lib.grid == (N, N, N) and lib.npw == orc.npw
        if x is None:
            x = synth.draw_x0(7, 8, orc.npw, 3)
            ref = O.apply_H(orc, x)
        assert rel(_run(lib, x), ref) < tol, (N, prec)


# every FFT plan of every register grid size (each factorisation N = L R
# with the full and the compact plane, and the Stockham passes where the full
# plane fits), one band per batch and the default batch, against the oracle
# on the same grid; FP64 at 128 and 144 runs on compact planes only
@pytest.mark.parametrize("N", [16, 24, 32, 36, 48, 64, 72, 96, 128, 144])
def test_apply_h_every_fft_plan(N):
    import paper_2406_10765_gb300 as pw
    ecut = 4.0 if N < 24 else 8.0
    plans = pw.pw_fft_plans(N)
    assert plans and all(L * R == N and L & (L - 1) == 0 and L <= 32 for L, R in plans)
    x = None
    for prec, tol, csize in (("fp64", 1e-12, 16), ("mixed", 1e-5, 8)):
        lib, orc, _ = cells("Si", 1, ecut, grid=(N, N, N), precision=prec)
        if x is None:
            x = synth.draw_x0(7, 8, orc.npw, 3)
            ref = O.apply_H(orc, x)
        full_fits = N * (N + 1) * csize <= 227 * 1024
        assert pw.pw_cell_get_fft_plan(lib.h, prec)[0:2] == plans[0]
        assert pw.pw_cell_get_fft_plan(lib.h, prec)[3] == (not full_fits)
        cands = [(L, R, cp) for L, R in plans for cp in (False, True) if full_fits or cp]
        if full_fits:
            cands.append((0, 0, False))
        else:
            # the full plane does not fit in shared memory in this precision
            with pytest.raises(pw.PwError):
                pw.pw_cell_set_fft_plan(lib.h, *plans[0], precision=prec)
            with pytest.raises(pw.PwError):
                pw.pw_cell_set_fft_plan(lib.h, 0, 0, precision=prec)
        for L, R, cp in cands:
            for batch in (1, 0):
                pw.pw_cell_set_fft_plan(lib.h, L, R, batch, precision=prec, compact=cp)
                got = pw.pw_cell_get_fft_plan(lib.h, prec)
                assert got[:2] == (L, R) and got[3] == cp
                assert rel(_run(lib, x), ref) < tol, (N, prec, L, R, cp, batch)
    with pytest.raises(pw.PwError):
        pw.pw_cell_set_fft_plan(lib.h, 3, N // 3 + 1, precision="mixed")
    with pytest.raises(pw.PwError):
        pw.pw_cell_set_fft_plan(lib.h, 0, 0, precision="mixed", compact=True)


def test_fft_autotune_si64():
    # the autotuner times every candidate plan of the 64-atom cell (grid 48)
    # and leaves the fastest set; H psi still matches the oracle
    import paper_2406_10765_gb300 as pw
    lib, orc, _ = cells("Si", 2, 10.0, precision="mixed")
    r = pw.pw_cell_autotune_fft(lib.h, 64, precision="mixed")
    ncand_min = 2 * len(pw.pw_fft_plans(lib.grid[0])) + 1
    assert r.ncand >= ncand_min
    assert 0 < r.ms_best <= r.ms_default
    assert pw.pw_cell_get_fft_plan(lib.h, "mixed") == (r.best.L, r.best.R, r.best.batch_bytes,
                                                      bool(r.best.compact))
    x = synth.draw_x0(3, 64, orc.npw, 4)
    assert rel(_run(lib, x), O.apply_H(orc, x)) < 1e-5


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("mixed", 1e-5)])
def test_projectors_on_the_fly(prec, tol):
    # beta regenerated in atom chunks (the 512-atom cell needs several 256 MB
    # chunks) gives the same H psi as the resident projectors and the oracle
    import paper_2406_10765_gb300 as pw
    lib, orc, _ = cells("Si", 4, 10.0, precision=prec)
    x = synth.draw_x0(21, 512, orc.npw, 12)
    stored = _run(lib, x)
    pw.pw_cell_set_projectors(lib.h, True)
    otf = _run(lib, x)
    for j in (0, 11):
        ref = O.apply_H(orc, x[:, j:j + 1])[:, 0]
        assert rel(otf[:, j], ref) < tol
    assert rel(otf, stored) < (1e-13 if prec == "fp64" else 1e-6)
    # no-allocation entry refuses a cell without resident projectors
    from paper_2406_10765_gb300 import binding as B
    psi = to_dev(x[:, :2])
    out = torch.empty_like(psi)
    assert B._apply_na(lib.h, B._dptr(psi), orc.npw, 2, B._dptr(out), B._stream(None)) == B.PW_ERR_ARG
    pw.pw_cell_set_projectors(lib.h, False)
    assert rel(_run(lib, x), stored) < (1e-15 if prec == "fp64" else 1e-12)


def test_apply_h_si1728_sampled():
    # the 1,728-atom cell (npw 251,967, grid 128^3, 6,912 projectors) with
    # projectors generated on the fly, on sampled bands against the oracle's
    # operator (its projectors formed 64 atoms at a time): mixed precision,
    # and FP64 on the compact x-y plane (the full FP64 plane does not fit in
    # shared memory at 128^2)
    import paper_2406_10765_gb300 as pw
    ci = synth.cell_inputs("Si", 6, 0)
    x = synth.draw_x0(0, 1728, 251967, 3)
    got = {}
    for prec in ("mixed", "fp64"):
        lib = pw.Cell(ci["L"], ci["tau"], ci["depth"], ci["dkb"], 8.0, precision=prec)
        assert lib.npw == 251967 and lib.grid == (128, 128, 128)
        pw.pw_cell_set_projectors(lib.h, True)
        if prec == "fp64":
            assert pw.pw_cell_get_fft_plan(lib.h, "fp64")[3]      # compact plane
        got[prec] = _run(lib, x)
    Ls = np.full(3, float(ci["L"]) if np.ndim(ci["L"]) == 0 else ci["L"][0])
    m = O.sphere(8.0, Ls)
    assert np.array_equal(lib.m, m)
    Ns = (128, 128, 128)
    V = O.vloc_grid(Ls, Ns, ci["tau"], ci["depth"], 1.2)
    orc = O.Cell(Ls=Ls, Ns=Ns, ecut=8.0, m=m, kin=O.kinetic(m, Ls), V=V,
                 beta=np.zeros((m.shape[0], 0), complex), D=np.zeros(0))
    ref = orc.kin[:, None] * x + O.apply_local(orc, x)
    D = np.asarray(ci["dkb"], float).reshape(-1)
    for a0 in range(0, len(ci["tau"]), 64):
        b = O.projectors(m, Ls, ci["tau"][a0:a0 + 64], 1.2)
        ref += b @ (D[4 * a0:4 * a0 + b.shape[1], None] * (b.conj().T @ x))
    assert rel(got["mixed"], ref) < 1e-5
    assert rel(got["fp64"], ref) < 1e-12
