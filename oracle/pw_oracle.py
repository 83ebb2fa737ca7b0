"""Plain FP64 CPU oracle for one block-eigensolver step of plane-wave
Kohn-Sham DFT with a fixed potential.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this module: only tests/, __graft_entry__.smoke() and the
cpu_baseline / reference legs of bench.py use it.  It shares no code with the
CUDA library (no kernels, headers, tables or generators); both sides are fed
the same seeded inputs from synth.py, which holds none of the method's
arithmetic.

Everything is float64 / complex128, written as the plain definition with numpy
and scipy library primitives (FFT, matmul, Cholesky, Hermitian eigensolver)
as single steps, and no blocking or reordering beyond the definition.

Every function here is pinned to something other than itself in
tests/test_oracle_pins.py (brute force, closed forms, invariants, textbook
special cases); tests/test_oracle_mutants.py plants mistakes in each
function's source and checks that the pins fail.

The problem (Sec. II-A, Eq. 1): H X = X Lambda for the lowest nb eigenpairs of
the plane-wave Hamiltonian, in Hartree atomic units,

  H_{GG'} = 1/2 |G|^2 delta_{GG'} + Vt((m - m') mod N)
            + sum_{a,i} beta_{ai}(G) D_{ai} conj(beta_{ai}(G'))

with G = 2 pi m / L on the sphere 1/2 |G|^2 <= Ecut (Sec. II-A), Vt the grid
Fourier coefficients of the local potential, and beta the Kleinman-Bylander
projectors (the pseudopotential application of Sec. III-A).  The iterative
solver is LOBPCG, one of the inner eigensolvers named in Sec. II-A; its step
is H*Psi (FFT based, Sec. II-B column scheme), the subspace matrices
S = Psi^H (H Psi) (Sec. II-B row scheme), and the small dense eigensolve
(Syevd, Sec. III-D), in the order of Knyazev's method.

Readings where the paper is silent (each is listed with its reason in the
design notes of the repository):
  * grid: smallest 2^a 3^b >= 1.5 * sqrt(2 Ecut) L / pi per axis (the paper's
    rule of Sec. II-A times 1.5);
  * FFT convention: psi(r_j) = sum_G c_G exp(i G.r_j), r_j = L j / N,
    forward transform scaled by N^-3, so the local term wraps modulo N;
  * local potential: sum over all periodic images of Gaussians
    d_a exp(-|r - tau_a - R|^2 / (2 sigma^2));
  * projectors: unit-norm Gaussian s and p_(x,y,z) functions of width r_p;
  * preconditioner: Teter-Payne-Allan on x = 1/2|G|^2 / E_kin(band);
  * Rayleigh-Ritz: Jacobi-scaled Gram, Cholesky; a pivot <= 1e-14 (relative)
    drops P for that step and retries;
  * active set: bands whose residual norm reached the tolerance leave W and P.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla

TWO_PI = 2.0 * math.pi


# --------------------------------------------------------------------------
# Cell, plane-wave sphere, FFT grid
# --------------------------------------------------------------------------

def grid_size_1d(ecut: float, L: float, factor: float = 1.5) -> int:
    """Smallest 2^a 3^b >= factor * sqrt(2 Ecut) L / pi  (Sec. II-A rule x 1.5)."""
    target = factor * math.sqrt(2.0 * ecut) * L / math.pi
    best = None
    p2 = 1
    while p2 < 4 * target + 8:
        p3 = p2
        while p3 < 4 * target + 8:
            if p3 >= target and (best is None or p3 < best):
                best = p3
            p3 *= 3
        p2 *= 2
    return int(best)


def sphere(ecut: float, Ls) -> np.ndarray:
    """Integer vectors m with 1/2 |2 pi m / L|^2 <= Ecut, lexicographic (mx, my, mz).

    Raises if any lattice point lies within 1e-9 Ha of the cutoff (the two
    sides of the boundary must not depend on rounding).
    """
    Ls = np.asarray(Ls, float)
    mmax = [int(math.floor(math.sqrt(2.0 * ecut) * L / TWO_PI)) + 1 for L in Ls]
    rng = [np.arange(-k, k + 1) for k in mmax]
    mx, my, mz = np.meshgrid(*rng, indexing="ij")
    m = np.stack([mx.ravel(), my.ravel(), mz.ravel()], axis=1)
    t = kinetic(m, Ls)
    if np.any(np.abs(t - ecut) < 1e-9):
        raise ValueError("a plane wave lies within 1e-9 Ha of Ecut")
    return m[t <= ecut].astype(np.int64)        # meshgrid 'ij' ravel is lexicographic


def kinetic(m, Ls) -> np.ndarray:
    """1/2 |G|^2 with G = 2 pi m / L."""
    g = TWO_PI * np.asarray(m, float) / np.asarray(Ls, float)[None, :]
    return 0.5 * np.sum(g * g, axis=1)


# --------------------------------------------------------------------------
# Local potential on the grid and its Fourier coefficients
# --------------------------------------------------------------------------

def vloc_grid(Ls, Ns, tau, depth, sigma, nimg: int = 3) -> np.ndarray:
    """V(r_j) = sum_a d_a sum_R exp(-|r_j - tau_a - R|^2 / (2 sigma^2)), array [jx, jy, jz].

    The lattice sum of a product of 1-D Gaussians factorises exactly into a
    product of 1-D periodic sums; the images |n| <= nimg (relative error of
    the dropped terms far below 1e-16 for the cells used) are kept.
    """
    Ls = np.asarray(Ls, float)
    tau = np.asarray(tau, float)
    V = np.zeros(tuple(Ns))
    per_axis = []
    for ax in range(3):
        r = Ls[ax] * np.arange(Ns[ax]) / Ns[ax]
        d = r[None, :] - tau[:, ax][:, None]                      # (natom, N)
        n = np.arange(-nimg, nimg + 1)
        dd = d[:, :, None] - n[None, None, :] * Ls[ax]
        per_axis.append(np.exp(-dd * dd / (2.0 * sigma * sigma)).sum(axis=2))
    for a in range(tau.shape[0]):
        V += depth[a] * np.einsum("i,j,k->ijk", per_axis[0][a], per_axis[1][a], per_axis[2][a])
    return V


def vloc_fourier(V: np.ndarray) -> np.ndarray:
    """Vt(k) = N^-3 sum_j V(r_j) exp(-i 2 pi k.j / N)  (grid Fourier coefficients)."""
    return np.fft.fftn(V) / V.size


# --------------------------------------------------------------------------
# Kleinman-Bylander projectors (Sec. III-A: per-atom pseudopotential data)
# --------------------------------------------------------------------------

def projectors(m, Ls, tau, rp: float) -> np.ndarray:
    """beta (npw, 4*natom): columns a*4 + (s, px, py, pz).

    beta_s(G)  = Omega^-1/2 N_s exp(-|G|^2 rp^2 / 2) exp(-i G.tau),  N_s^2 = 8 pi^1.5 rp^3
    beta_pa(G) = Omega^-1/2 N_p (-i) G_a exp(-|G|^2 rp^2 / 2) exp(-i G.tau), N_p^2 = 16 pi^1.5 rp^5
    (Fourier transforms of unit-norm Gaussian s and p functions of width rp.)
    """
    Ls = np.asarray(Ls, float)
    tau = np.asarray(tau, float)
    omega = float(np.prod(Ls))
    G = TWO_PI * np.asarray(m, float) / Ls[None, :]
    g2 = np.sum(G * G, axis=1)
    radial = np.exp(-0.5 * g2 * rp * rp) / math.sqrt(omega)
    ns = math.sqrt(8.0 * math.pi ** 1.5 * rp ** 3)
    npn = math.sqrt(16.0 * math.pi ** 1.5 * rp ** 5)
    natom = tau.shape[0]
    beta = np.empty((G.shape[0], 4 * natom), dtype=np.complex128)
    for a in range(natom):
        phase = np.exp(-1j * (G @ tau[a]))
        beta[:, 4 * a] = ns * radial * phase
        for k in range(3):
            beta[:, 4 * a + 1 + k] = npn * (-1j) * G[:, k] * radial * phase
    return beta


# --------------------------------------------------------------------------
# The Hamiltonian
# --------------------------------------------------------------------------

@dataclass
class Cell:
    Ls: np.ndarray
    Ns: tuple
    ecut: float
    m: np.ndarray
    kin: np.ndarray
    V: np.ndarray            # real-space local potential [jx, jy, jz]
    beta: np.ndarray         # (npw, nproj)
    D: np.ndarray            # (nproj,)
    extra: dict = field(default_factory=dict)

    @property
    def npw(self) -> int:
        return self.m.shape[0]


def make_cell(L, tau, depth, dkb, ecut, sigma=1.2, rp=1.2, grid=None, V=None) -> Cell:
    """Build the oracle's cell.  `L` is a scalar (cubic) or 3 lengths."""
    Ls = np.broadcast_to(np.asarray(L, float), (3,)).copy()
    m = sphere(ecut, Ls)
    Ns = tuple(int(g) for g in grid) if grid is not None else \
        tuple(grid_size_1d(ecut, Ls[i]) for i in range(3))
    if V is None:
        V = vloc_grid(Ls, Ns, tau, depth, sigma)
    beta = projectors(m, Ls, tau, rp)
    D = np.asarray(dkb, float).reshape(-1)
    return Cell(Ls=Ls, Ns=Ns, ecut=ecut, m=m, kin=kinetic(m, Ls), V=V, beta=beta, D=D)


def to_real_space(cell: Cell, c: np.ndarray) -> np.ndarray:
    """psi(r_j) = sum_G c_G exp(i G.r_j) for each column of c -> array [jx, jy, jz, band]."""
    N = cell.Ns
    nb = c.shape[1]
    grid = np.zeros(N + (nb,), dtype=np.complex128)
    idx = tuple((cell.m[:, k] % N[k]) for k in range(3))
    grid[idx] = c
    return np.fft.ifftn(grid, axes=(0, 1, 2)) * (N[0] * N[1] * N[2])


def to_sphere(cell: Cell, f: np.ndarray) -> np.ndarray:
    """f_G = N^-3 sum_j f(r_j) exp(-i G.r_j) on the sphere (each band)."""
    N = cell.Ns
    F = np.fft.fftn(f, axes=(0, 1, 2)) / (N[0] * N[1] * N[2])
    idx = tuple((cell.m[:, k] % N[k]) for k in range(3))
    return F[idx]


def apply_local(cell: Cell, c: np.ndarray) -> np.ndarray:
    """(V psi)_G through the grid: G -> r, multiply by V(r), r -> G."""
    psi_r = to_real_space(cell, c)
    return to_sphere(cell, cell.V[..., None] * psi_r)


def apply_nonlocal(cell: Cell, c: np.ndarray) -> np.ndarray:
    """sum_{ai} beta_ai D_ai (beta_ai^H c)  (Sec. III-A, applied to all bands at once)."""
    B = cell.beta.conj().T @ c
    return cell.beta @ (cell.D[:, None] * B)


def apply_H(cell: Cell, c: np.ndarray) -> np.ndarray:
    """H c for a block c (npw, nb): kinetic + local + nonlocal."""
    c = np.asarray(c, dtype=np.complex128)
    if c.ndim == 1:
        return apply_H(cell, c[:, None])[:, 0]
    return cell.kin[:, None] * c + apply_local(cell, c) + apply_nonlocal(cell, c)


def dense_H(cell: Cell) -> np.ndarray:
    """The explicit npw x npw Hamiltonian matrix from its definition."""
    Vt = vloc_fourier(cell.V)
    N = cell.Ns
    dm = cell.m[:, None, :] - cell.m[None, :, :]
    Hl = Vt[dm[..., 0] % N[0], dm[..., 1] % N[1], dm[..., 2] % N[2]]
    H = Hl + np.diag(cell.kin) + (cell.beta * cell.D[None, :]) @ cell.beta.conj().T
    return H


def dense_eigs(cell: Cell, nb: int | None = None):
    """Eigenpairs of the dense H (LAPACK Hermitian eigensolver)."""
    H = dense_H(cell)
    if nb is None:
        return sla.eigh(H)
    return sla.eigh(H, subset_by_index=[0, nb - 1])


# --------------------------------------------------------------------------
# LOBPCG (Knyazev 2001), one step at a time
# --------------------------------------------------------------------------

class CholeskyBreakdown(Exception):
    pass


def tpa(x: np.ndarray) -> np.ndarray:
    """Teter-Payne-Allan (1989) preconditioner polynomial ratio."""
    p = 27.0 + x * (18.0 + x * (12.0 + 8.0 * x))
    return p / (p + 16.0 * x ** 4)


def band_kinetic(cell: Cell, X: np.ndarray) -> np.ndarray:
    """E_kin(band) = sum_G 1/2|G|^2 |x_G|^2 / sum_G |x_G|^2."""
    w = np.abs(X) ** 2
    return (cell.kin[:, None] * w).sum(axis=0) / w.sum(axis=0)


def precondition(cell: Cell, X: np.ndarray, R: np.ndarray) -> np.ndarray:
    """W = K(R): per band, K(x) with x = 1/2|G|^2 / E_kin(band)."""
    ek = band_kinetic(cell, X)
    return tpa(cell.kin[:, None] / ek[None, :]) * R


def rayleigh_ritz(S: np.ndarray, HS: np.ndarray, nb: int, piv_tol: float = 1e-14):
    """Lowest nb Ritz pairs of the pencil (S^H H S, S^H S).

    Gram G = S^H S and A = S^H (H S); Jacobi scaling d = diag(G)^-1/2;
    Cholesky d G d = L L^H (breakdown if a pivot <= piv_tol * max pivot of
    the scaled matrix); At = L^-1 (d A d) L^-H; eigh(At) -> (theta, Y);
    coefficients C = d L^-H Y[:, :nb].
    """
    G = S.conj().T @ S
    A = S.conj().T @ HS
    G = 0.5 * (G + G.conj().T)
    A = 0.5 * (A + A.conj().T)
    d = 1.0 / np.sqrt(np.real(np.diag(G)))
    Gs = d[:, None] * G * d[None, :]
    As = d[:, None] * A * d[None, :]
    try:
        L = sla.cholesky(Gs, lower=True)
    except np.linalg.LinAlgError as e:
        raise CholeskyBreakdown(str(e))
    piv = np.real(np.diag(L)) ** 2
    if piv.min() <= piv_tol * np.real(np.diag(Gs)).max():
        raise CholeskyBreakdown("small pivot")
    T = sla.solve_triangular(L, As, lower=True)                  # L^-1 As
    At = sla.solve_triangular(L, T.conj().T, lower=True).conj().T  # (L^-1 (L^-1 As)^H)^H
    At = 0.5 * (At + At.conj().T)
    theta, Y = sla.eigh(At)
    C = d[:, None] * sla.solve_triangular(L.conj().T, Y[:, :nb], lower=False)
    return theta[:nb], C


@dataclass
class LobpcgState:
    X: np.ndarray
    HX: np.ndarray
    lam: np.ndarray
    P: np.ndarray | None = None
    HP: np.ndarray | None = None
    active: np.ndarray | None = None      # bool (nb,): columns still iterated
    it: int = 0
    resid: np.ndarray | None = None
    dropped_p: int = 0


def lobpcg_init(cell: Cell, X0: np.ndarray, nb: int | None = None) -> LobpcgState:
    """Orthonormalise the random block and take its Ritz vectors (Cholesky QR + RR)."""
    nb = X0.shape[1] if nb is None else nb
    HX0 = apply_H(cell, X0)
    lam, C = rayleigh_ritz(X0, HX0, nb)
    return LobpcgState(X=X0 @ C, HX=HX0 @ C, lam=lam, active=np.ones(nb, bool))


def residual(st: LobpcgState):
    """R = HX - X Lambda and the 2-norms of its columns."""
    R = st.HX - st.X * st.lam[None, :]
    return R, np.sqrt(np.sum(np.abs(R) ** 2, axis=0))


def lobpcg_step(cell: Cell, st: LobpcgState, tol_lock: float = 0.0) -> LobpcgState:
    """One LOBPCG iteration (Knyazev 2001).

    Active set: column i stays active while ||r_i|| > tol_lock (once inactive
    it stays inactive); only active columns enter W and P.
    R = HX - X Lambda; W = K R_act; HW = H W; S = [X, W, P_act];
    Rayleigh-Ritz -> C; X' = S C; P' = [0, W, P_act] C (Hetmaniuk-Lehoucq),
    and the same combinations of the H blocks, so H is applied once (to W).
    """
    nb = st.X.shape[1]
    R, rn = residual(st)
    act = (rn > tol_lock) & (st.active if st.active is not None else True)
    W = precondition(cell, st.X, R)[:, act]
    HW = apply_H(cell, W)
    dropped = 0
    blocks, hblocks = [st.X, W], [st.HX, HW]
    if st.P is not None:
        blocks.append(st.P[:, act])
        hblocks.append(st.HP[:, act])
    S = np.hstack(blocks)
    HS = np.hstack(hblocks)
    try:
        lam, C = rayleigh_ritz(S, HS, nb)
    except CholeskyBreakdown:
        if st.P is None:
            raise
        k = nb + int(act.sum())
        S, HS = S[:, :k], HS[:, :k]
        lam, C = rayleigh_ritz(S, HS, nb)
        dropped = 1
    X = S @ C
    HX = HS @ C
    P = S[:, nb:] @ C[nb:]
    HP = HS[:, nb:] @ C[nb:]
    return LobpcgState(X=X, HX=HX, lam=lam, P=P, HP=HP, active=act, it=st.it + 1,
                       resid=rn, dropped_p=st.dropped_p + dropped)


def eigsolve(cell: Cell, X0: np.ndarray, tol: float = 1e-8, maxit: int = 200):
    """Iterate until max_i ||H x_i - theta_i x_i|| <= tol (columns below tol
    are locked).  Returns (lam, X, iters, resid)."""
    st = lobpcg_init(cell, X0)
    for _ in range(maxit + 1):
        _, rn = residual(st)
        if rn.max() <= tol:
            return st.lam, st.X, st.it, rn
        if st.it >= maxit:
            break
        st = lobpcg_step(cell, st, tol_lock=tol)
    _, rn = residual(st)
    return st.lam, st.X, st.it, rn


# --------------------------------------------------------------------------
# Density (Sec. II-A): rho(r) = sum_j |psi_j(r)|^2
# --------------------------------------------------------------------------

def density(cell: Cell, X: np.ndarray, occ: np.ndarray | None = None) -> np.ndarray:
    psi = to_real_space(cell, X)
    w = np.ones(X.shape[1]) if occ is None else occ
    return np.einsum("xyzb,b->xyz", np.abs(psi) ** 2, w)


# --------------------------------------------------------------------------
# Self-consistent field with a model V_Hxc (the outer loop of Sec. II-A; the
# paper fixes no exchange-correlation functional, so the model is Hartree
# plus Slater/Dirac exchange)
# --------------------------------------------------------------------------

def grid_gvectors(Ls, Ns) -> np.ndarray:
    """|G|^2 on the full FFT grid, G = 2 pi k / L with k the signed index
    (0 .. N/2, then negative), array [kx, ky, kz]."""
    ks = [np.fft.fftfreq(Ns[a]) * Ns[a] for a in range(3)]
    g = [TWO_PI * ks[a] / Ls[a] for a in range(3)]
    return g[0][:, None, None] ** 2 + g[1][None, :, None] ** 2 + g[2][None, None, :] ** 2


def hartree_potential(Ls, Ns, n: np.ndarray) -> np.ndarray:
    """Periodic solution of lap V_H = -4 pi (n - <n>): V_H(r_j) = sum_{G != 0}
    4 pi n~(G) / |G|^2 exp(i G.r_j), n~ the grid Fourier coefficients."""
    nt = np.fft.fftn(n) / n.size
    g2 = grid_gvectors(Ls, Ns)
    vt = np.zeros_like(nt)
    nz = g2 > 0
    vt[nz] = 4.0 * math.pi * nt[nz] / g2[nz]
    return np.real(np.fft.ifftn(vt) * n.size)


def slater_exchange(n: np.ndarray) -> np.ndarray:
    """Dirac/Slater exchange potential v_x = -(3 n / pi)^(1/3) (n >= 0)."""
    return -np.cbrt(3.0 * np.maximum(n, 0.0) / math.pi)


def electron_density(cell: Cell, X: np.ndarray, occ: np.ndarray) -> np.ndarray:
    """n(r_j) = Omega^-1 sum_b occ_b |psi_b(r_j)|^2 (unit-norm coefficient
    columns), so sum_j n_j Omega / N^3 = sum_b occ_b."""
    return density(cell, X, occ) / float(np.prod(cell.Ls))


def scf(cell0: Cell, nocc: int, fill: float = 2.0, mix: float = 0.3, niter: int = 8,
        hxc_scale: float = 1.0):
    """Linear density mixing: n_in <- (1 - mix) n_in + mix n_out, starting
    from n_in = 0.  Iteration k: V = V_loc + hxc_scale (V_H + v_x)[n_in], the
    lowest nocc eigenpairs of the dense H (LAPACK), n_out from them with
    occupation `fill`.  Returns per iteration (eigenvalues, n_in, n_out)."""
    n_in = np.zeros(cell0.Ns)
    hist = []
    occ = np.full(nocc, fill)
    for _ in range(niter):
        V = cell0.V + hxc_scale * (hartree_potential(cell0.Ls, cell0.Ns, n_in) + slater_exchange(n_in))
        cell = Cell(Ls=cell0.Ls, Ns=cell0.Ns, ecut=cell0.ecut, m=cell0.m, kin=cell0.kin, V=V,
                    beta=cell0.beta, D=cell0.D)
        w, X = dense_eigs(cell, nocc)
        n_out = electron_density(cell, X, occ)
        hist.append((w, n_in.copy(), n_out))
        n_in = (1.0 - mix) * n_in + mix * n_out
    return hist
