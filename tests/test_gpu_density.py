"""Electron density rho(r) = sum_b w_b |psi_b(r)|^2 on the FFT grid (the
quantity the self-consistent loop of Sec. II-A forms from the wavefunctions)
against the oracle's density, through the C ABI."""
import numpy as np
import pytest

import synth
from oracle import pw_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from gpu_util import cells, to_dev  # noqa: E402


def _rho(lib, x, occ=None):
    import paper_2406_10765_gb300 as pw
    psi = to_dev(x)
    w = torch.from_numpy(np.asarray(occ, float)).cuda() if occ is not None else None
    r = pw.pw_density(lib.h, psi, w)
    torch.cuda.synchronize()
    return r.cpu().numpy().transpose(2, 1, 0)      # (z, y, x) -> (x, y, z) as the oracle


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("species,n,ecut,grid,nb", [
    ("Si", 1, 10.0, None, 24),            # 24^3: register line FFTs
    ("C", 1, 8.0, None, 18),              # 16^3
    ("Si", 1, 6.0, (18, 27, 16), 7),      # non-cubic: Stockham passes
])
def test_density_fp64_matches_oracle(species, n, ecut, grid, nb):
    lib, orc, _ = cells(species, n, ecut, grid=grid)
    x = synth.draw_x0(11, 8 * n ** 3, orc.npw, nb)
    occ = np.linspace(2.0, 0.5, nb)
    got = _rho(lib, x, occ)
    ref = O.density(orc, x, occ)
    assert got.shape == ref.shape
    assert _rel(got, ref) < 1e-12
    # sum rule (Parseval): sum_j rho_j = N^3 sum_b w_b ||c_b||^2
    N3 = np.prod(orc.Ns)
    assert abs(got.sum() - N3 * (occ * (np.abs(x) ** 2).sum(axis=0)).sum()) < 1e-10 * got.sum()


def test_density_mixed_precision():
    lib, orc, _ = cells("Si", 1, 10.0, precision="mixed")
    x = synth.draw_x0(12, 8, orc.npw, 16)
    assert _rel(_rho(lib, x), O.density(orc, x)) < 1e-5


def test_density_si512_batches_and_determinism():
    # full-size grid (96^3), bands spanning two L2 batches; unit weights
    lib, orc, _ = cells("Si", 4, 10.0)
    x = synth.draw_x0(13, 512, orc.npw, 20)
    got = _rho(lib, x)
    assert _rel(got, O.density(orc, x)) < 1e-12
    assert np.array_equal(got, _rho(lib, x))       # bitwise repeatable


def test_density_zero_bands_and_errors():
    import paper_2406_10765_gb300 as pw
    from paper_2406_10765_gb300 import binding as B
    import ctypes as ct
    lib, orc, _ = cells("C", 1, 8.0)
    rho = torch.full(tuple(reversed(lib.grid)), 7.0, dtype=torch.float64, device="cuda")
    x = to_dev(synth.draw_x0(1, 8, orc.npw, 2))
    st = B._stream(None)
    assert B._density(lib.h, B._dptr(x), orc.npw, 0, ct.c_void_p(), B._dptr(rho), st) == 0
    torch.cuda.synchronize()
    assert float(rho.abs().max()) == 0.0
    assert B._density(lib.h, B._dptr(x), orc.npw - 1, 2, ct.c_void_p(), B._dptr(rho), st) == B.PW_ERR_ARG
    assert B._density(lib.h, B._dptr(x), orc.npw, 2, ct.c_void_p(), ct.c_void_p(), st) == B.PW_ERR_ARG
