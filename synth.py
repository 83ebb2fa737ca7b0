"""Seeded synthetic inputs for the plane-wave eigensolver workloads.

This module only *generates inputs*: atomic positions of diamond-structure
Si / C supercells and the seeded random draws (Gaussian-well depths,
Kleinman-Bylander coefficients, the random starting block).  It holds none of
the method's arithmetic (no sphere, grid, potential, projector or solver).
Both the oracle and the CUDA library are fed from here; the library also has
its own SplitMix64 for requests that carry only a seed, and the tests check
that the two agree.

Random numbers: SplitMix64 (Steele, Lea, Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), used counter-style: draw i of
seed s is mix(s + (i+1)*0x9E3779B97F4A7C15), i.e. the i-th output of the
sequential generator started at state s.  Uniform doubles are the top 53 bits
times 2**-53.

Stream layout for a cell of `natom` atoms (counter offsets):
  depth[a]          -> i = a                       (a < natom)
  dkb[a, k]         -> i = natom + 4*a + k         (k = s, px, py, pz)
  X0[g, j] real     -> i = 5*natom + 2*(j*npw + g)
  X0[g, j] imag     -> i = 5*natom + 2*(j*npw + g) + 1
"""
from __future__ import annotations

import numpy as np

SI_A = 10.26          # bohr, Si diamond cubic lattice constant
C_A = 6.74            # bohr, C diamond cubic lattice constant
SIGMA = 1.2           # bohr, width of the Gaussian local wells
RP = 1.2              # bohr, radial width of the Gaussian KB projectors
DEPTH_MEAN = -1.0     # Ha
DEPTH_SPREAD = 0.1    # Ha (uniform in mean +- spread)
DKB_LO, DKB_HI = 0.5, 1.5   # Ha

# fractional positions of the 8-atom diamond cubic basis
DIAMOND_BASIS = np.array([
    [0.00, 0.00, 0.00], [0.00, 0.50, 0.50], [0.50, 0.00, 0.50], [0.50, 0.50, 0.00],
    [0.25, 0.25, 0.25], [0.25, 0.75, 0.75], [0.75, 0.25, 0.75], [0.75, 0.75, 0.25],
])

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, idx) -> np.ndarray:
    """uint64 draws number `idx` (array of non-negative ints) of stream `seed`."""
    idx = np.asarray(idx, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (idx + np.uint64(1)) * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, idx) -> np.ndarray:
    """Uniform doubles in [0, 1) from counter positions `idx`."""
    return (splitmix64(seed, idx) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def diamond_supercell(a: float, n: int):
    """Cubic n x n x n supercell of the 8-atom diamond cell.

    Returns (L, tau) with L = n*a (bohr) and tau (8 n^3, 3) Cartesian bohr,
    ordered by cell index (ix, iy, iz) lexicographic, then basis atom.
    """
    cells = np.array([(i, j, k) for i in range(n) for j in range(n) for k in range(n)], float)
    frac = (cells[:, None, :] + DIAMOND_BASIS[None, :, :]).reshape(-1, 3)
    return n * a, frac * a


def draw_depths(seed: int, natom: int) -> np.ndarray:
    u = uniform01(seed, np.arange(natom))
    return DEPTH_MEAN + DEPTH_SPREAD * (2.0 * u - 1.0)


def draw_dkb(seed: int, natom: int) -> np.ndarray:
    """(natom, 4) diagonal KB coefficients D_s, D_px, D_py, D_pz in [0.5, 1.5) Ha."""
    u = uniform01(seed, natom + np.arange(4 * natom))
    return (DKB_LO + (DKB_HI - DKB_LO) * u).reshape(natom, 4)


def draw_x0(seed: int, natom: int, npw: int, nb: int) -> np.ndarray:
    """Random starting block (npw, nb) complex128, Fortran (column-major) order.

    Entry (g, j) = (u1 - 1/2) + i (u2 - 1/2).
    """
    base = 5 * natom
    j = np.arange(nb, dtype=np.uint64)[:, None]
    g = np.arange(npw, dtype=np.uint64)[None, :]
    k = np.uint64(base) + np.uint64(2) * (j * np.uint64(npw) + g)
    re = uniform01(seed, k) - 0.5
    im = uniform01(seed, k + np.uint64(1)) - 0.5
    return np.asfortranarray((re + 1j * im).T)


def cell_inputs(species: str, n: int, seed: int = 0):
    """Diamond Si or C supercell with its seeded depths and KB coefficients.

    Returns dict(L, tau, depth, dkb, sigma, rp).
    """
    a = {"Si": SI_A, "C": C_A}[species]
    L, tau = diamond_supercell(a, n)
    natom = tau.shape[0]
    return dict(L=L, tau=tau, depth=draw_depths(seed, natom), dkb=draw_dkb(seed, natom),
                sigma=SIGMA, rp=RP)


def periodic_depths(species: str, n: int, seed: int = 0):
    """Supercell whose depths / KB coefficients repeat those of the 8-atom cell
    drawn with `seed` (used for the supercell-folding checks)."""
    base = cell_inputs(species, 1, seed)
    L, tau = diamond_supercell({"Si": SI_A, "C": C_A}[species], n)
    reps = n ** 3
    return dict(L=L, tau=tau, depth=np.tile(base["depth"], reps),
                dkb=np.tile(base["dkb"], (reps, 1)), sigma=SIGMA, rp=RP)


# Poisson serving stream -------------------------------------------------------

def serving_requests(nreq: int, rate_per_s: float, seed: int = 12345):
    """Request list for the serving workload.

    Each request: species Si or C (50/50), n in {1, 2, 3}, Ecut ~ U[8, 12] Ha,
    nbands = 1.125 * (2 * natom) (rounded), seed = request id, and a Poisson
    arrival time (exponential gaps of mean 1/rate).
    """
    idx = np.arange(nreq, dtype=np.uint64) * np.uint64(4)
    u_sp = uniform01(seed, idx)
    u_n = uniform01(seed, idx + np.uint64(1))
    u_e = uniform01(seed, idx + np.uint64(2))
    u_t = uniform01(seed, idx + np.uint64(3))
    gaps = -np.log1p(-u_t) / rate_per_s
    t = np.cumsum(gaps) - gaps[0]
    out = []
    for r in range(nreq):
        species = "Si" if u_sp[r] < 0.5 else "C"
        n = 1 + int(min(2, np.floor(3 * u_n[r])))
        natom = 8 * n ** 3
        out.append(dict(id=r, species=species, n=n, ecut=8.0 + 4.0 * float(u_e[r]),
                        nbands=int(round(1.125 * 2 * natom)), seed=r, t_arrival=float(t[r])))
    return out
