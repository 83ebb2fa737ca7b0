"""SCF outer loop with the model V_Hxc (Sec. II-A; Hartree + Slater exchange)
against the oracle's loop, through the C ABI."""
import numpy as np
import pytest

import synth
from oracle import pw_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from gpu_util import cells, to_dev, rel  # noqa: E402


def _grid(a):       # (x, y, z) numpy -> CUDA (z, y, x)
    return torch.from_numpy(np.ascontiguousarray(a.transpose(2, 1, 0))).cuda()


def _host(t):       # CUDA (z, y, x) -> numpy (x, y, z)
    return t.cpu().numpy().transpose(2, 1, 0)


@pytest.mark.parametrize("species,ecut,grid", [("Si", 10.0, None), ("Si", 6.0, (18, 27, 16))])
def test_hxc_potential_matches_oracle(species, ecut, grid):
    import paper_2406_10765_gb300 as pw
    lib, orc, _ = cells(species, 1, ecut, grid=grid)
    rng = np.random.default_rng(3)
    n = 0.01 + 0.05 * rng.random(orc.Ns)
    v = _host(pw.pw_hxc_potential(lib.h, _grid(n)))
    ref = O.hartree_potential(orc.Ls, orc.Ns, n) + O.slater_exchange(n)
    assert np.abs(v - ref).max() < 1e-12 * np.abs(ref).max()


def test_set_hxc_changes_h_and_restores():
    import paper_2406_10765_gb300 as pw
    lib, orc, _ = cells("Si", 1, 10.0)
    rng = np.random.default_rng(4)
    vx = 0.2 * rng.standard_normal(orc.Ns)
    x = synth.draw_x0(5, 8, orc.npw, 6)
    pw.pw_cell_set_hxc(lib.h, _grid(vx))
    psi, out = to_dev(x), pw.new_block(orc.npw, 6)
    pw.pw_apply_H(lib.h, psi, out)
    torch.cuda.synchronize()
    orc2 = O.Cell(Ls=orc.Ls, Ns=orc.Ns, ecut=orc.ecut, m=orc.m, kin=orc.kin, V=orc.V + vx,
                  beta=orc.beta, D=orc.D)
    assert rel(out.cpu().numpy(), O.apply_H(orc2, x)) < 1e-12
    pw.pw_cell_set_hxc(lib.h, None)
    pw.pw_apply_H(lib.h, psi, out)
    torch.cuda.synchronize()
    assert rel(out.cpu().numpy(), O.apply_H(orc, x)) < 1e-12


def test_scf_iterations_match_oracle():
    # C-8 model insulator (8 doubly occupied bands, gap 0.21 Ha): the same
    # six mixing iterations on both sides
    import paper_2406_10765_gb300 as pw
    lib, orc, _ = cells("C", 1, 8.0)
    eig, n_out, rep, st = pw.pw_scf(lib.h, 12, 8, mix=0.5, maxiter=6, tol=0.0, eig_tol=1e-11,
                                    raise_noconv=False)
    assert st == pw.PW_ERR_NOCONV and rep.iters == 6
    h = O.scf(orc, 8, mix=0.5, niter=6)
    w_ref, _, nout_ref = h[-1]
    assert np.abs(eig[:8] - w_ref).max() < 1e-9
    assert np.abs(_host(n_out) - nout_ref).max() < 1e-8 * np.abs(nout_ref).max()
    assert abs(rep.max_dn - np.abs(nout_ref - h[-1][1]).max()) < 1e-8


def test_scf_converges_to_the_oracle_fixed_point():
    import paper_2406_10765_gb300 as pw
    lib, orc, _ = cells("C", 1, 8.0)
    eig, n_out, rep, st = pw.pw_scf(lib.h, 12, 8, mix=0.5, maxiter=40, tol=1e-7, eig_tol=1e-11)
    assert st == pw.PW_OK and rep.max_dn <= 1e-7
    h = O.scf(orc, 8, mix=0.5, niter=rep.iters)
    assert np.abs(_host(n_out) - h[-1][2]).max() < 1e-6
    # electron count of the converged density: 16
    n = _host(n_out)
    assert abs(n.sum() * np.prod(orc.Ls) / n.size - 16.0) < 1e-9
    pw.pw_cell_set_hxc(lib.h, None)


def test_scf_argument_errors():
    import paper_2406_10765_gb300 as pw
    lib, _, _ = cells("C", 1, 8.0)
    for kw in (dict(nbands=4, nocc=8), dict(nbands=8, nocc=8, mix=0.0), dict(nbands=8, nocc=8, maxiter=0)):
        with pytest.raises(pw.PwError):
            pw.pw_scf(lib.h, **kw)
