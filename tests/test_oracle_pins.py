"""Pins for the FP64 oracle against things other than itself: brute force on
tiny inputs, closed forms, invariants and special cases that reduce to a
textbook result.  Each test names the part of the method it guards."""
import itertools
import math

import numpy as np
import pytest
import scipy.optimize as sopt

import synth
from oracle import pw_oracle as O

TWO_PI = 2 * math.pi


def _cell(species="Si", n=1, ecut=10.0, seed=0, **kw):
    ci = synth.cell_inputs(species, n, seed)
    return O.make_cell(ci["L"], ci["tau"], ci["depth"], ci["dkb"], ecut, **kw), ci


# ---------------------------------------------------------------- inputs ----

def test_splitmix64_published_values():
    # first outputs of SplitMix64 seeded with 0 (Steele, Lea, Flood 2014)
    z = synth.splitmix64(0, np.arange(3))
    assert [int(v) for v in z] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_synth_ranges():
    ci = synth.cell_inputs("Si", 2, 7)
    assert ci["tau"].shape == (64, 3)
    assert np.all((ci["depth"] >= -1.1) & (ci["depth"] < -0.9))
    assert np.all((ci["dkb"] >= 0.5) & (ci["dkb"] < 1.5))
    # the 8 basis atoms of the diamond cell: nearest-neighbour distance sqrt(3)/4 a
    L, tau = synth.diamond_supercell(synth.SI_A, 1)
    d = np.linalg.norm(tau[:, None] - tau[None], axis=2) + 1e9 * np.eye(8)
    assert abs(d.min() - math.sqrt(3) / 4 * synth.SI_A) < 1e-12


# ---------------------------------------------------------- sphere, grid ----

def _brute_sphere(ecut, L):
    R = int(math.sqrt(2 * ecut) * L / TWO_PI) + 2
    out = []
    for mx in range(-R, R + 1):
        for my in range(-R, R + 1):
            for mz in range(-R, R + 1):
                g2 = (TWO_PI / L) ** 2 * (mx * mx + my * my + mz * mz)
                if 0.5 * g2 <= ecut:
                    out.append((mx, my, mz))
    return np.array(out)


@pytest.mark.parametrize("species,ecut", [("Si", 10.0), ("C", 8.0), ("Si", 4.0)])
def test_sphere_brute_force(species, ecut):
    L = {"Si": synth.SI_A, "C": synth.C_A}[species]
    m = O.sphere(ecut, [L] * 3)
    ref = _brute_sphere(ecut, L)          # loops already run in lexicographic order
    assert m.shape == ref.shape and np.array_equal(m, ref)


def test_sphere_counts_and_volume():
    # Npw of the three workload cells, and the lattice-point count of a ball
    for n, ecut, want in [(1, 10.0, 1647), (4, 10.0, 104415), (6, 8.0, 251967)]:
        L = n * synth.SI_A
        npw = O.sphere(ecut, [L] * 3).shape[0]
        assert npw == want
        R = math.sqrt(2 * ecut) * L / TWO_PI
        assert abs(npw / (4 / 3 * math.pi * R ** 3) - 1) < 0.05


def test_grid_rule():
    smooth = sorted(2 ** a * 3 ** b for a in range(10) for b in range(7))
    for ecut, L in [(10.0, 10.26), (10.0, 41.04), (8.0, 61.56), (8.0, 6.74), (12.0, 30.78)]:
        target = 1.5 * math.sqrt(2 * ecut) * L / math.pi
        assert O.grid_size_1d(ecut, L) == next(s for s in smooth if s >= target)
    assert [O.grid_size_1d(10, 10.26), O.grid_size_1d(10, 41.04), O.grid_size_1d(8, 61.56)] == [24, 96, 128]
    # the grid must hold the sphere without aliasing: 2 mmax < N
    for ecut, L in [(10.0, 10.26), (8.0, 6.74)]:
        m = O.sphere(ecut, [L] * 3)
        assert 2 * np.abs(m).max() < O.grid_size_1d(ecut, L)
    # each axis of a cell with three different lengths gets its own grid
    cell = O.make_cell(np.array([6.0, 9.0, 13.0]), np.array([[0.3, 1.1, 2.0]]), np.array([-1.0]),
                       np.array([[0.7, 0.9, 1.1, 1.3]]), 6.0)
    assert cell.Ns == (12, 16, 24)        # 1.5 sqrt(2 Ecut) L / pi = 9.9, 14.9, 21.5
    for k in range(3):
        assert 2 * np.abs(cell.m[:, k]).max() < cell.Ns[k]


# ------------------------------------------------------------------ FFT ----

def _tiny_cell(Ns=(6, 9, 8), Ls=(5.0, 7.0, 6.0), ecut=3.0, V=None):
    tau = np.array([[0.3, 1.1, 2.0], [2.9, 4.0, 0.7]])
    depth = np.array([-1.0, -0.95])
    dkb = np.array([[0.7, 0.9, 1.1, 1.3], [0.6, 0.8, 1.0, 1.2]])
    return O.make_cell(np.array(Ls), tau, depth, dkb, ecut, grid=Ns, V=V)


def test_fft_convention_brute_force():
    cell = _tiny_cell()
    rng = np.random.default_rng(1)
    c = rng.standard_normal((cell.npw, 2)) + 1j * rng.standard_normal((cell.npw, 2))
    psi = O.to_real_space(cell, c)
    G = TWO_PI * cell.m / cell.Ls
    for j in [(0, 0, 0), (1, 2, 3), (5, 8, 7), (3, 0, 4)]:
        r = cell.Ls * np.array(j) / np.array(cell.Ns)
        direct = (np.exp(1j * (G @ r))[:, None] * c).sum(axis=0)
        assert np.allclose(psi[j], direct, atol=1e-12)
    # forward: f_G = N^-3 sum_j f(r_j) exp(-i G.r_j)
    f = rng.standard_normal(cell.Ns) + 0j
    fg = O.to_sphere(cell, f[..., None])[:, 0]
    pts = np.array(list(itertools.product(*[range(n) for n in cell.Ns])))
    rj = pts * (cell.Ls / np.array(cell.Ns))
    for g in [0, 5, cell.npw - 1]:
        direct = (f[tuple(pts.T)] * np.exp(-1j * (rj @ G[g]))).sum() / np.prod(cell.Ns)
        assert abs(fg[g] - direct) < 1e-12


def test_parseval_and_roundtrip():
    cell, _ = _cell("Si", 1, 10.0)
    rng = np.random.default_rng(2)
    c = rng.standard_normal((cell.npw, 3)) + 1j * rng.standard_normal((cell.npw, 3))
    psi = O.to_real_space(cell, c)
    n3 = np.prod(cell.Ns)
    assert np.allclose((np.abs(psi) ** 2).sum(axis=(0, 1, 2)), n3 * (np.abs(c) ** 2).sum(axis=0), rtol=1e-13)
    assert np.abs(O.to_sphere(cell, psi) - c).max() < 1e-13


# ------------------------------------------------------ local potential ----

def test_vloc_direct_image_sum():
    Ls = np.array([5.0, 6.0, 5.5])
    Ns = (8, 6, 5)
    tau = np.array([[0.3, 1.1, 2.0], [4.6, 5.9, 0.1]])
    depth = np.array([-1.0, -0.9])
    V = O.vloc_grid(Ls, Ns, tau, depth, 1.2)
    for j in [(0, 0, 0), (7, 5, 4), (3, 2, 1)]:
        r = Ls * np.array(j) / np.array(Ns)
        tot = 0.0
        for a in range(2):
            for R in itertools.product(range(-4, 5), repeat=3):
                d = r - tau[a] - Ls * np.array(R)
                tot += depth[a] * math.exp(-(d @ d) / (2 * 1.2 ** 2))
        assert abs(V[j] - tot) < 1e-13


def test_vloc_cell_average():
    # mean of a periodised Gaussian over the cell = its integral / Omega
    cell, ci = _cell("Si", 1, 10.0)
    omega = np.prod(cell.Ls)
    want = ci["depth"].sum() * (2 * math.pi * ci["sigma"] ** 2) ** 1.5 / omega
    assert abs(cell.V.mean() - want) < 1e-12 * abs(want)


def test_vloc_fourier_brute_force():
    cell = _tiny_cell()
    Vt = O.vloc_fourier(cell.V)
    pts = np.array(list(itertools.product(*[range(n) for n in cell.Ns])))
    for k in [(0, 0, 0), (1, 2, 3), (5, 1, 7)]:
        ph = np.exp(-2j * math.pi * (pts @ (np.array(k) / np.array(cell.Ns))))
        assert abs(Vt[k] - (cell.V[tuple(pts.T)] * ph).sum() / len(pts)) < 1e-14


# ----------------------------------------------------------- projectors ----

def test_projector_normalisation():
    # unit real-space norm: sum_G |beta(G)|^2 -> 1 when the sphere holds the
    # whole Gaussian (its periodic self-overlap is exp(-L^2/(4 rp^2)) ~ 1e-8)
    L = synth.SI_A
    m = O.sphere(60.0, [L] * 3)
    tau = np.array([[1.0, 2.0, 3.0]])
    beta = O.projectors(m, [L] * 3, tau, 1.2)
    norms = (np.abs(beta) ** 2).sum(axis=0)
    assert np.allclose(norms, 1.0, atol=1e-6)
    ov = beta.conj().T @ beta
    assert np.abs(ov - np.diag(np.diag(ov))).max() < 1e-10   # s, px, py, pz orthogonal


# -------------------------------------------------------- whole operator ----

def test_free_electron_shells():
    # V = 0, D = 0: eigenvalues are 1/2|G|^2; Si cell unit (2 pi / a)^2 / 2
    cell, _ = _cell("Si", 1, 10.0)
    cell.V = np.zeros(cell.Ns)
    cell.D = np.zeros_like(cell.D)
    w = np.linalg.eigvalsh(O.dense_H(cell))
    unit = 0.5 * (TWO_PI / synth.SI_A) ** 2
    assert abs(unit - 0.187514) < 1e-6
    shells = [(0, 1), (1, 6), (2, 12), (3, 8), (4, 6), (5, 24), (6, 24), (8, 12)]
    want = np.concatenate([[s * unit] * g for s, g in shells])
    assert np.abs(w[:len(want)] - want).max() < 1e-12
    # LOBPCG reaches the same 19 lowest (the block ends on a shell boundary)
    X0 = synth.draw_x0(0, 8, cell.npw, 19)
    lam, X, it, rn = O.eigsolve(cell, X0, tol=1e-9, maxit=200)
    assert np.abs(lam - want[:19]).max() < 1e-12


def test_constant_potential_shift():
    cell, _ = _cell("C", 1, 8.0)
    w0 = np.linalg.eigvalsh(O.dense_H(cell))
    cell.V = cell.V + 0.37
    w1 = np.linalg.eigvalsh(O.dense_H(cell))
    assert np.abs(w1 - w0 - 0.37).max() < 1e-12


def test_rank_one_secular_equation():
    # V = 0, one atom with only an s projector: 1 + D sum |b_G|^2 / (t_G - e) = 0
    L = synth.C_A
    ecut = 8.0
    tau = np.array([[0.4, 1.3, 2.2]])
    dkb = np.array([[0.8, 0.0, 0.0, 0.0]])
    cell = O.make_cell(L, tau, np.array([0.0]), dkb, ecut)
    cell.V = np.zeros(cell.Ns)
    w = np.linalg.eigvalsh(O.dense_H(cell))
    t = cell.kin
    b2 = np.abs(cell.beta[:, 0]) ** 2
    shells = np.unique(np.round(t, 10))
    wt = np.array([b2[np.abs(t - s) < 1e-9].sum() for s in shells])
    deg = np.array([(np.abs(t - s) < 1e-9).sum() for s in shells])
    D = 0.8
    f = lambda e: 1 + D * np.sum(wt / (shells - e))
    roots = [sopt.brentq(f, shells[i] + 1e-13, shells[i + 1] - 1e-13, xtol=1e-15)
             for i in range(len(shells) - 1)]
    hi = shells[-1] + D * wt.sum() + 1.0
    roots.append(sopt.brentq(f, shells[-1] + 1e-13, hi, xtol=1e-15))
    # each shell keeps deg-1 copies of its energy; the secular roots are the rest
    want = np.sort(np.concatenate([np.repeat(shells, deg - 1), roots]))
    assert np.abs(w - want).max() < 1e-10


def test_hermiticity_and_dense_agreement():
    cell, _ = _cell("Si", 1, 10.0)
    rng = np.random.default_rng(3)
    x = rng.standard_normal((cell.npw, 2)) + 1j * rng.standard_normal((cell.npw, 2))
    Hx = O.apply_H(cell, x)
    a = np.vdot(x[:, 0], Hx[:, 1])
    b = np.vdot(x[:, 1], Hx[:, 0])
    assert abs(a - np.conj(b)) < 1e-13 * abs(a)
    H = O.dense_H(cell)
    assert np.abs(H - H.conj().T).max() < 1e-15
    assert np.linalg.norm(H @ x - Hx) < 1e-13 * np.linalg.norm(Hx)


def test_grid_shift_and_permutation_invariance():
    ci = synth.cell_inputs("C", 1, 4)
    ecut = 8.0
    base = O.make_cell(ci["L"], ci["tau"], ci["depth"], ci["dkb"], ecut)
    w0 = np.linalg.eigvalsh(O.dense_H(base))
    N = np.array(base.Ns)
    shift = ci["L"] * np.array([3, -5, 7]) / N
    moved = O.make_cell(ci["L"], ci["tau"] + shift, ci["depth"], ci["dkb"], ecut)
    assert np.abs(np.linalg.eigvalsh(O.dense_H(moved)) - w0).max() < 1e-12
    p = np.random.default_rng(5).permutation(8)
    perm = O.make_cell(ci["L"], ci["tau"][p], ci["depth"][p], ci["dkb"][p], ecut)
    assert np.abs(np.linalg.eigvalsh(O.dense_H(perm)) - w0).max() < 1e-12


def test_supercell_folding():
    # with depths repeating every cell and grid n*N_cell, an eigenvector of the
    # 8-atom cell, placed on G' = G_cell (c'_{n m} = c_m), is an eigenvector of
    # the n^3-cell Hamiltonian with the same eigenvalue
    ecut = 10.0
    small = synth.periodic_depths("Si", 1, 3)
    big = synth.periodic_depths("Si", 2, 3)
    cs = O.make_cell(small["L"], small["tau"], small["depth"], small["dkb"], ecut)
    cb = O.make_cell(big["L"], big["tau"], big["depth"], big["dkb"], ecut)
    assert cb.Ns == tuple(2 * n for n in cs.Ns)
    w, v = O.dense_eigs(cs, 6)
    # normalisation: beta scales with Omega^-1/2; the nonlocal term
    # sum_a beta beta^H has 8x the atoms and 1/8 the weight per atom
    index = {tuple(mm): i for i, mm in enumerate(cb.m)}
    c = np.zeros((cb.npw, 6), complex)
    for i, mm in enumerate(cs.m):
        c[index[tuple(2 * mm)], :] = v[i, :]
    Hc = O.apply_H(cb, c)
    assert np.abs(Hc - c * w[None, :]).max() < 1e-12


def _cyclic_jacobi_eigvals(H, tol=1e-14, max_sweeps=30):
    """Eigenvalues of a Hermitian matrix by Jacobi's method: sweeps of 2 x 2
    unitary rotations, each zeroing one off-diagonal pair, in the parallel
    round-robin ordering (n/2 disjoint pairs per round, n - 1 rounds per
    sweep), with the inner angle |theta| <= pi/4, until the off-diagonal
    Frobenius norm is below tol ||H||_F.  For the pair (p, q) with
    h_pq = |h_pq| e^{i phi}: tan 2 theta = 2 |h_pq| / (h_pp - h_qq) and the
    rotation's columns are (cos, e^{-i phi} sin), (-sin, e^{-i phi} cos)."""
    A = np.array(H, dtype=np.complex128)
    n = A.shape[0]
    m = n + (n % 2)                       # one idle index when n is odd
    fro = np.linalg.norm(A)
    order = np.arange(m)
    for _ in range(max_sweeps):
        if np.linalg.norm(A - np.diag(np.diag(A))) <= tol * fro:
            return np.sort(np.real(np.diag(A)))
        for _ in range(m - 1):
            P, Q = order[: m // 2], order[::-1][: m // 2]
            keep = (P < n) & (Q < n)
            P, Q = P[keep], Q[keep]
            a, d, b = np.real(A[P, P]), np.real(A[Q, Q]), A[P, Q]
            ab = np.abs(b)
            with np.errstate(divide="ignore", invalid="ignore"):
                th = 0.5 * np.arctan(np.where(ab > 0, 2 * ab / (a - d), 0.0))
                ph = np.where(ab > 0, np.conj(b) / ab, 1.0)
            c, s = np.cos(th), np.sin(th)
            g11, g12, g21, g22 = c, -s, ph * s, ph * c
            AP, AQ = A[:, P].copy(), A[:, Q].copy()
            A[:, P], A[:, Q] = AP * g11 + AQ * g21, AP * g12 + AQ * g22
            RP, RQ = A[P, :].copy(), A[Q, :].copy()
            A[P, :] = np.conj(g11)[:, None] * RP + np.conj(g21)[:, None] * RQ
            A[Q, :] = np.conj(g12)[:, None] * RP + np.conj(g22)[:, None] * RQ
            order = np.concatenate([order[:1], order[-1:], order[1:-1]])
    raise AssertionError("Jacobi sweeps did not converge")


def test_dense_eigs_against_cyclic_jacobi():
    # the oracle's dense diagonalisation (which the LOBPCG pins compare
    # with) against Jacobi's method on a C-8 cell of 203 plane waves
    cell, _ = _cell("C", 1, 6.0)
    assert cell.npw == 203
    w, _ = O.dense_eigs(cell)
    wj = _cyclic_jacobi_eigvals(O.dense_H(cell))
    assert np.abs(w - wj).max() < 1e-12


def test_lobpcg_vs_dense_and_bounds():
    cell, _ = _cell("C", 1, 8.0, seed=2)
    nb = 18
    w, _ = O.dense_eigs(cell, nb + 1)
    X0 = synth.draw_x0(2, 8, cell.npw, nb)
    lam, X, it, rn = O.eigsolve(cell, X0, tol=1e-9, maxit=300)
    assert rn.max() <= 1e-9
    assert np.abs(lam - w[:nb]).max() < 1e-12
    # Weyl: each Ritz value within its residual norm of an eigenvalue
    assert np.all(np.abs(lam - w[:nb]) <= rn + 1e-14)
    assert np.abs(X.conj().T @ X - np.eye(nb)).max() < 1e-12


def test_kato_temple_bound_on_a_loose_solve():
    # Ritz pairs stopped at max residual 1e-3: each Ritz value is within
    # ||r||^2 / delta of its eigenvalue (Kato-Temple; delta = distance to the
    # rest of the spectrum), far inside the first-order Weyl bound ||r||
    cell, _ = _cell("C", 1, 8.0, seed=2)
    nb = 18
    w = np.linalg.eigvalsh(O.dense_H(cell))
    lam, X, it, rn = O.eigsolve(cell, synth.draw_x0(2, 8, cell.npw, nb), tol=1e-3, maxit=300)
    assert rn.max() <= 1e-3 and rn.max() > 1e-5
    for i in range(nb):
        j = np.argmin(np.abs(w - lam[i]))
        assert j == i
        delta = np.abs(np.delete(w, j) - lam[i]).min()
        assert abs(lam[i] - w[j]) <= rn[i] ** 2 / delta
        assert lam[i] >= w[j] - 1e-12          # Ritz values bound from above


def test_lobpcg_seed_independence():
    cell, _ = _cell("C", 1, 8.0, seed=1)
    a = O.eigsolve(cell, synth.draw_x0(11, 8, cell.npw, 12), tol=1e-9)[0]
    b = O.eigsolve(cell, synth.draw_x0(12, 8, cell.npw, 12), tol=1e-9)[0]
    assert np.abs(a - b).max() < 1e-12


def test_tpa_closed_form():
    assert O.tpa(np.array([0.0]))[0] == 1.0
    assert abs(O.tpa(np.array([1.0]))[0] - 65.0 / 81.0) < 1e-15
    x = np.array([1e4])
    assert abs(O.tpa(x)[0] * 2 * x[0] - 1) < 1e-3      # ~ 8x^3 / 16x^4
    xs = np.linspace(0, 10, 101)
    assert np.all(np.diff(O.tpa(xs)) < 0)


def test_rayleigh_ritz_breakdown_and_solution():
    rng = np.random.default_rng(4)
    S = rng.standard_normal((50, 4)) + 1j * rng.standard_normal((50, 4))
    Hm = rng.standard_normal((50, 50))
    Hm = Hm + Hm.T
    with pytest.raises(O.CholeskyBreakdown):
        O.rayleigh_ritz(np.hstack([S, S[:, :1]]), Hm @ np.hstack([S, S[:, :1]]), 2)
    lam, C = O.rayleigh_ritz(S, Hm @ S, 4)
    # the Ritz values of the pencil solve the generalized problem
    import scipy.linalg as sla
    ref = sla.eigh(S.conj().T @ Hm @ S, S.conj().T @ S, eigvals_only=True)
    assert np.abs(lam - ref).max() < 1e-10
    X = S @ C
    assert np.abs(X.conj().T @ X - np.eye(4)).max() < 1e-12


def test_rayleigh_ritz_pivot_threshold():
    """The drop test fires on a scaled pivot <= 1e-14 even where the Cholesky
    itself succeeds.  The last pivot of the Jacobi-scaled Gram is the squared
    distance of the last unit column from the span of the others, computed
    here by least squares: at 3e-15 the step must report a breakdown, at
    3e-13 it must not."""
    import scipy.linalg as sla
    rng = np.random.default_rng(7)
    A = rng.standard_normal((60, 5)) + 1j * rng.standard_normal((60, 5))
    A /= np.linalg.norm(A, axis=0)
    b = rng.standard_normal(60) + 1j * rng.standard_normal(60)
    b -= A @ np.linalg.lstsq(A, b, rcond=None)[0]            # b orthogonal to span(A)
    Hm = rng.standard_normal((60, 60))
    Hm = Hm + Hm.T
    for piv, breaks in [(3e-15, True), (3e-13, False)]:
        # last column a_1 + e b: distance^2 / norm^2 = e^2 |b|^2 / (1 + e^2 |b|^2)
        e = math.sqrt(piv / (1 - piv)) / np.linalg.norm(b)
        S = np.hstack([A, (A[:, 1] + e * b)[:, None]])
        u = S[:, -1] / np.linalg.norm(S[:, -1])
        dist2 = np.linalg.norm(u - A @ np.linalg.lstsq(A, u, rcond=None)[0]) ** 2
        assert abs(dist2 / piv - 1) < 1e-2
        G = S.conj().T @ S
        d = 1 / np.sqrt(np.real(np.diag(G)))
        sla.cholesky(d[:, None] * G * d[None, :], lower=True)   # factorises either way
        if breaks:
            with pytest.raises(O.CholeskyBreakdown):
                O.rayleigh_ritz(S, Hm @ S, 2)
        else:
            O.rayleigh_ritz(S, Hm @ S, 2)


def _rr_pencil(S, HS, nb):
    """Lowest nb eigenvalues of the pencil (S^H H S, S^H S) by scipy's
    generalized Hermitian solver: a route that shares nothing with the
    oracle's Jacobi scaling, Cholesky and triangular solves."""
    import scipy.linalg as sla
    A = S.conj().T @ HS
    B = S.conj().T @ S
    return sla.eigh(0.5 * (A + A.conj().T), 0.5 * (B + B.conj().T), eigvals_only=True)[:nb]


def _w_from_definition(cell, st):
    """W written out: R = H X - X Lambda, each column scaled by the TPA ratio
    p / (p + 16 x^4), p = 27 + 18 x + 12 x^2 + 8 x^3, x = 1/2|G|^2 / E_kin."""
    R = O.apply_H(cell, st.X) - st.X * st.lam[None, :]
    ek = (cell.kin[:, None] * np.abs(st.X) ** 2).sum(0) / (np.abs(st.X) ** 2).sum(0)
    x = cell.kin[:, None] / ek[None, :]
    p = 27 + 18 * x + 12 * x ** 2 + 8 * x ** 3
    return p / (p + 16 * x ** 4) * R


def _outside(V, Q):
    """Relative size of the part of V's columns outside span(Q)."""
    c, *_ = np.linalg.lstsq(Q, V, rcond=None)
    return np.abs(V - Q @ c).max() / np.abs(V).max()


def test_lobpcg_step_drops_p_on_breakdown():
    """Cholesky breakdown inside the step (Knyazev's method with the pivot
    reading): with P inside span(X) the Gram of [X, W, P] is singular, so the
    step must retry on [X, W] alone.  Pinned against a generalized
    eigensolve of that pencil, with W formed from the definition."""
    cell, _ = _cell("Si", 1, 10.0)
    nb = 6
    st = O.lobpcg_init(cell, synth.draw_x0(3, 8, cell.npw, nb))
    rng = np.random.default_rng(11)
    Q = rng.standard_normal((nb, nb)) + 1j * rng.standard_normal((nb, nb))
    st.P, st.HP = st.X @ Q, st.HX @ Q
    nxt = O.lobpcg_step(cell, st)
    assert nxt.dropped_p == 1
    W = _w_from_definition(cell, st)
    S = np.hstack([st.X, W])
    ref = _rr_pencil(S, O.apply_H(cell, S), nb)
    assert np.abs(nxt.lam - ref).max() < 1e-10
    # Ritz values of a larger space can only fall (Cauchy interlacing)
    assert np.all(nxt.lam <= st.lam + 1e-12)
    # the retried block is orthonormal and solves the projected problem
    assert np.abs(nxt.X.conj().T @ nxt.X - np.eye(nb)).max() < 1e-12
    Rn = O.apply_H(cell, nxt.X) - nxt.X * nxt.lam[None, :]
    assert np.abs(S.conj().T @ Rn).max() < 1e-9 * np.abs(S).max() * np.abs(Rn).max() * cell.npw
    # P' is the [0, W] part only: orthogonal complement test against span(X)
    assert nxt.P.shape == (cell.npw, nb)


def test_lobpcg_step_keeps_p_when_it_is_independent():
    """The same state with a P outside span([X, W]) keeps P (no drop): the
    step equals the generalized eigensolve of the full pencil [X, W, P]."""
    cell, _ = _cell("Si", 1, 10.0)
    nb = 6
    st = O.lobpcg_init(cell, synth.draw_x0(3, 8, cell.npw, nb))
    P = synth.draw_x0(5, 8, cell.npw, nb)
    st.P, st.HP = P, O.apply_H(cell, P)
    nxt = O.lobpcg_step(cell, st)
    assert nxt.dropped_p == 0
    R = st.HX - st.X * st.lam[None, :]
    W = O.precondition(cell, st.X, R)
    S = np.hstack([st.X, W, P])
    ref = _rr_pencil(S, O.apply_H(cell, S), nb)
    assert np.abs(nxt.lam - ref).max() < 1e-10


def test_lobpcg_step_direction_update():
    """The new direction carries no X component (Knyazev's method in the
    Hetmaniuk-Lehoucq form): P' lies in span([W, P]) and X' - P' in
    span(X), so X' = X C_X + P'.  The H blocks follow the same
    combinations: HX' = H X' and HP' = H P'."""
    cell, _ = _cell("Si", 1, 10.0)
    nb = 6
    st = O.lobpcg_init(cell, synth.draw_x0(3, 8, cell.npw, nb))
    P = synth.draw_x0(5, 8, cell.npw, nb)
    st.P, st.HP = P, O.apply_H(cell, P)
    nxt = O.lobpcg_step(cell, st)
    W = _w_from_definition(cell, st)
    assert _outside(nxt.P, np.hstack([W, P])) < 1e-10
    assert _outside(nxt.X - nxt.P, st.X) < 1e-10
    # and P' is a real direction, not a copy of X'
    assert _outside(nxt.P, st.X) > 1e-3
    assert np.abs(nxt.HX - O.apply_H(cell, nxt.X)).max() < 1e-10 * np.abs(nxt.HX).max()
    assert np.abs(nxt.HP - O.apply_H(cell, nxt.P)).max() < 1e-10 * np.abs(nxt.HP).max()


def test_lobpcg_init_is_the_ritz_block_of_the_start():
    """The first block: orthonormal, H X carried exactly, and the Ritz values
    of span(X0), i.e. the generalized eigenvalues of (X0^H H X0, X0^H X0),
    with X^H H X diagonal."""
    cell, _ = _cell("Si", 1, 10.0)
    nb = 6
    X0 = synth.draw_x0(3, 8, cell.npw, nb)
    st = O.lobpcg_init(cell, X0)
    assert np.abs(st.X.conj().T @ st.X - np.eye(nb)).max() < 1e-12
    assert np.abs(st.HX - O.apply_H(cell, st.X)).max() < 1e-10 * np.abs(st.HX).max()
    assert np.abs(st.lam - _rr_pencil(X0, O.apply_H(cell, X0), nb)).max() < 1e-10
    assert np.abs(st.X.conj().T @ st.HX - np.diag(st.lam)).max() < 1e-10
    assert _outside(st.X, X0) < 1e-12


def test_lobpcg_init_breakdown_on_dependent_start():
    """A start block with two equal columns has a singular Gram: the initial
    Cholesky QR reports a breakdown (the library's PW_ERR_CHOL)."""
    cell, _ = _cell("C", 1, 8.0)
    x0 = synth.draw_x0(2, 8, cell.npw, 4)
    x0[:, 3] = x0[:, 1]
    with pytest.raises(O.CholeskyBreakdown):
        O.lobpcg_init(cell, x0)


def test_density_sum_rule():
    cell, _ = _cell("C", 1, 8.0)
    w, v = O.dense_eigs(cell, 4)
    rho = O.density(cell, v)
    assert abs(rho.mean() - 4.0) < 1e-12       # Parseval: each band contributes 1


def test_free_electron_golden_table():
    here = __import__("os").path.dirname(__file__)
    rows = np.loadtxt(here + "/golden/free_electron_si.txt", dtype=int)
    L = synth.SI_A
    m = O.sphere(10.0, [L] * 3)
    n2 = (m ** 2).sum(axis=1)
    for s, g in rows:
        assert (n2 == s).sum() == g


# ---- model V_Hxc and the SCF loop -------------------------------------------

def test_hartree_single_mode_closed_form():
    # n = A cos(G.r) with G = 2 pi (2, -1, 3) / L: V_H = 4 pi A cos(G.r) / |G|^2
    Ls = np.array([7.0, 8.0, 9.0])
    Ns = (16, 18, 24)
    k = np.array([2, -1, 3])
    G = 2 * np.pi * k / Ls
    r = [Ls[a] * np.arange(Ns[a]) / Ns[a] for a in range(3)]
    phase = G[0] * r[0][:, None, None] + G[1] * r[1][None, :, None] + G[2] * r[2][None, None, :]
    n = 0.37 * np.cos(phase) + 0.05                   # the constant has no potential
    V = O.hartree_potential(Ls, Ns, n)
    ref = 4 * np.pi * 0.37 * np.cos(phase) / (G @ G)
    assert np.abs(V - ref).max() < 1e-12


def test_hartree_sine_mode_sign():
    # an odd mode fixes the direction of both transforms: n = A sin(G.r)
    # gives V_H = 4 pi A sin(G.r) / |G|^2 (a flipped exponent flips its sign)
    Ls = np.array([7.0, 8.0, 9.0])
    Ns = (16, 18, 24)
    G = 2 * np.pi * np.array([1, 3, -2]) / Ls
    r = [Ls[a] * np.arange(Ns[a]) / Ns[a] for a in range(3)]
    phase = G[0] * r[0][:, None, None] + G[1] * r[1][None, :, None] + G[2] * r[2][None, None, :]
    V = O.hartree_potential(Ls, Ns, 0.21 * np.sin(phase))
    assert np.abs(V - 4 * np.pi * 0.21 * np.sin(phase) / (G @ G)).max() < 1e-12


def test_hartree_superposition_and_zero_mean():
    rng = np.random.default_rng(0)
    Ls, Ns = np.array([6.0, 6.0, 6.0]), (12, 12, 12)
    a, b = rng.random(Ns), rng.random(Ns)
    Va, Vb = O.hartree_potential(Ls, Ns, a), O.hartree_potential(Ls, Ns, b)
    assert np.abs(O.hartree_potential(Ls, Ns, 2 * a - b) - (2 * Va - Vb)).max() < 1e-12
    assert abs(Va.mean()) < 1e-13


def test_slater_exchange_uniform_gas():
    # Dirac exchange potential of the uniform gas at r_s = 2: n = 3 / (4 pi r_s^3),
    # v_x = -(3 n / pi)^(1/3) = -(9 / (4 pi^2))^(1/3) / r_s
    rs = 2.0
    n = np.full((2, 2, 2), 3.0 / (4 * np.pi * rs ** 3))
    ref = -((9.0 / (4.0 * np.pi ** 2)) ** (1.0 / 3.0)) / rs
    assert np.abs(O.slater_exchange(n) - ref).max() < 1e-15


def test_scf_reduces_to_fixed_potential_and_counts_electrons():
    ci = synth.cell_inputs("Si", 1, 0)
    cell = O.make_cell(ci["L"], ci["tau"], ci["depth"], ci["dkb"], 6.0)
    # no V_Hxc: every iteration is the fixed-potential eigenproblem
    h = O.scf(cell, 8, niter=2, hxc_scale=0.0)
    w0, _ = O.dense_eigs(cell, 8)
    assert np.abs(h[1][0] - w0).max() < 1e-12
    # electron count: sum_j n_j Omega / N^3 = 2 x 8
    n_out = h[0][2]
    assert abs(n_out.sum() * np.prod(cell.Ls) / n_out.size - 16.0) < 1e-10


def test_scf_mixing_converges_to_a_fixed_point():
    # the synthetic wells give a gapped model insulator with 8 doubly
    # occupied bands (gap 0.21 Ha for C-8); linear mixing contracts to the
    # self-consistent density
    ci = synth.cell_inputs("C", 1, 0)
    cell = O.make_cell(ci["L"], ci["tau"], ci["depth"], ci["dkb"], 8.0)
    h = O.scf(cell, 8, mix=0.5, niter=16)
    d = [np.abs(n_out - n_in).max() for _, n_in, n_out in h]
    assert d[-1] < 1e-4 * d[0]
    assert all(d[k + 2] < d[k] for k in range(len(d) - 2))
    # the limit is a fixed point of the Kohn-Sham map: the lowest 8 bands of
    # V_loc + V_H[n] + v_x[n], doubly occupied, give back n
    n = h[-1][2]
    V = cell.V + O.hartree_potential(cell.Ls, cell.Ns, n) + O.slater_exchange(n)
    ks = O.make_cell(ci["L"], ci["tau"], ci["depth"], ci["dkb"], 8.0, V=V)
    _, X = O.dense_eigs(ks, 8)
    n2 = O.electron_density(ks, X, np.full(8, 2.0))
    assert np.abs(n2 - n).max() < 10 * d[-1]
    # and not of the bare potential
    _, X0 = O.dense_eigs(cell, 8)
    assert np.abs(O.electron_density(cell, X0, np.full(8, 2.0)) - n).max() > 1e3 * d[-1]


def test_scf_linear_mixing_is_a_geometric_series():
    # with no V_Hxc every iteration sees the same potential, so n_out is the
    # same density n* each time and n_in after k iterations is the partial
    # sum alpha sum_{i<k} (1 - alpha)^i n* = (1 - (1 - alpha)^k) n*
    ci = synth.cell_inputs("C", 1, 0)
    cell = O.make_cell(ci["L"], ci["tau"], ci["depth"], ci["dkb"], 8.0)
    alpha = 0.3
    h = O.scf(cell, 8, mix=alpha, niter=4, hxc_scale=0.0)
    nstar = h[0][2]
    for k, (_, n_in, n_out) in enumerate(h):
        assert np.abs(n_out - nstar).max() < 1e-12 * np.abs(nstar).max()
        assert np.abs(n_in - (1 - (1 - alpha) ** k) * nstar).max() < 1e-12 * np.abs(nstar).max()
