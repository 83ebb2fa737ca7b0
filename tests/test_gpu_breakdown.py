"""The method's degenerate cases on the GPU, against the oracle: a Cholesky
breakdown inside the LOBPCG step (P dropped, the step retried on [X, W]), a
singular start block (PW_ERR_CHOL) and NaN inputs (PW_ERR_NUMERIC).  Every
failure is made on the host (the inputs); nothing here faults the GPU."""
import numpy as np
import pytest

import synth
from oracle import pw_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from gpu_util import cells, to_dev  # noqa: E402


def _state(precision):
    import paper_2406_10765_gb300 as pw
    lib, orc, _ = cells("Si", 1, 10.0)
    nb = 8
    x0 = synth.draw_x0(3, 8, orc.npw, nb)
    s = pw.pw_solver_create(lib.h, nb, tol=0.0, x0=x0, precision=precision)
    return pw, lib, orc, x0, nb, s


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 1e-4)])
def test_step_drops_p_inside_span_x(precision, tol):
    pw, lib, orc, x0, nb, s = _state(precision)
    rng = np.random.default_rng(11)
    Q = rng.standard_normal((nb, nb)) + 1j * rng.standard_normal((nb, nb))
    # P = X Q lies inside span(X): the Gram of [X, W, P] is singular
    X = pw.new_block(lib.npw, nb)
    pw.pw_solver_block(s, X)
    pw.pw_solver_set_p(s, X.cpu().numpy() @ Q)
    rep = pw.pw_subspace_step(lib.h, s)
    assert rep.dropped_p == 1 and rep.nsub == 2 * nb
    e, _ = pw.pw_solver_eigs(s, nb)
    # the oracle's step from the same state (its own Ritz vectors, P = X Q)
    st = O.lobpcg_init(orc, x0)
    st.P, st.HP = st.X @ Q, st.HX @ Q
    nxt = O.lobpcg_step(orc, st)
    assert nxt.dropped_p == 1
    assert np.abs(e - nxt.lam).max() < tol, np.abs(e - nxt.lam).max()
    # the step after the retry has a P again and runs on [X, W, P]
    rep2 = pw.pw_subspace_step(lib.h, s)
    assert rep2.dropped_p == 0 and rep2.nsub == 3 * nb
    nxt2 = O.lobpcg_step(orc, nxt)
    e2, _ = pw.pw_solver_eigs(s, nb)
    assert np.abs(e2 - nxt2.lam).max() < tol
    pw.pw_solver_destroy(s)


def test_set_p_round_trip_and_independent_p_kept():
    pw, lib, orc, x0, nb, s = _state("fp64")
    P = synth.draw_x0(5, 8, orc.npw, nb)
    pw.pw_solver_set_p(s, P)
    out = pw.new_block(lib.npw, nb)
    assert pw.pw_solver_get_p(s, out)
    got = out.cpu().numpy()
    # stored with unit columns
    assert np.abs(got - P / np.linalg.norm(P, axis=0)).max() < 1e-14
    rep = pw.pw_subspace_step(lib.h, s)
    assert rep.dropped_p == 0 and rep.nsub == 3 * nb
    st = O.lobpcg_init(orc, x0)
    st.P, st.HP = P, O.apply_H(orc, P)
    nxt = O.lobpcg_step(orc, st)
    e, _ = pw.pw_solver_eigs(s, nb)
    assert np.abs(e - nxt.lam).max() < 1e-10
    pw.pw_solver_destroy(s)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_singular_start_block_reports_chol(precision):
    import paper_2406_10765_gb300 as pw
    lib, orc, _ = cells("C", 1, 8.0)
    x0 = synth.draw_x0(2, 8, orc.npw, 4)
    x0[:, 3] = x0[:, 1]
    with pytest.raises(O.CholeskyBreakdown):
        O.lobpcg_init(orc, x0)
    with pytest.raises(pw.PwError) as e:
        pw.pw_solver_create(lib.h, 4, tol=0.0, x0=x0, precision=precision)
    assert e.value.status == pw.PW_ERR_CHOL
    # the context is still usable: a good start block solves
    s = pw.pw_solver_create(lib.h, 4, tol=0.0, x0=synth.draw_x0(2, 8, orc.npw, 4), precision=precision)
    pw.pw_subspace_step(lib.h, s)
    pw.pw_solver_destroy(s)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_nan_start_block_reports_numeric(precision):
    import paper_2406_10765_gb300 as pw
    lib, orc, _ = cells("C", 1, 8.0)
    x0 = synth.draw_x0(2, 8, orc.npw, 4)
    x0[7, 2] = np.nan
    with pytest.raises(pw.PwError) as e:
        pw.pw_solver_create(lib.h, 4, tol=0.0, x0=x0, precision=precision)
    assert e.value.status == pw.PW_ERR_NUMERIC


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_nan_search_direction_reports_numeric_in_the_step(precision):
    pw, lib, orc, x0, nb, s = _state(precision)
    P = synth.draw_x0(5, 8, orc.npw, nb)
    P[11, 4] = np.inf
    pw.pw_solver_set_p(s, P)
    with pytest.raises(pw.PwError) as e:
        pw.pw_subspace_step(lib.h, s)
    assert e.value.status == pw.PW_ERR_NUMERIC
    pw.pw_solver_destroy(s)
