"""FP64-accurate tensor-core complex product (pw_zgemm_f64tc) against numpy's
complex128 product: every op combination, ragged shapes that span several
tiles, alpha/beta, wide dynamic range between rows, and the error bound
K 2^-53 max_k|a_ik| max_k|b_kj| per entry (the FP64 product bound's scale)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from gpu_util import to_dev  # noqa: E402


def _rand(rng, shape, spread=0.0):
    x = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    if spread:
        x *= np.exp2(rng.uniform(-spread, spread, size=(shape[0], 1)))
    return x


def _op(x, op):
    return x if op == "N" else x.conj().T


def _check(opA, opB, m, n, k, alpha=1.0, beta=0.0, spread=0.0, seed=0):
    import paper_2406_10765_gb300 as pw
    rng = np.random.default_rng(seed)
    A = _rand(rng, (m, k) if opA == "N" else (k, m), spread)
    B = _rand(rng, (k, n) if opB == "N" else (n, k), spread)
    C0 = _rand(rng, (m, n))
    got = pw.pw_zgemm_f64tc(opA, opB, to_dev(A), to_dev(B), to_dev(C0), alpha=alpha, beta=beta)
    torch.cuda.synchronize()
    got = got.cpu().numpy()
    oa, ob = _op(A, opA), _op(B, opB)
    ref = alpha * (oa @ ob) + beta * C0
    amax = np.abs(oa).max(axis=1)
    bmax = np.abs(ob).max(axis=0)
    scale = abs(alpha) * np.outer(amax, bmax) * 2 * k * 2.0 ** -53 + abs(beta) * np.abs(C0) * 2.0 ** -52
    err = np.abs(got - ref)
    assert np.all(np.isfinite(got))
    assert (err <= 4 * scale + 1e-300).all(), (err / scale).max()
    return err, scale


@pytest.mark.parametrize("opA,opB", [("N", "N"), ("C", "N"), ("N", "C"), ("C", "C")])
def test_f64tc_ops_ragged(opA, opB):
    _check(opA, opB, 300, 97, 211, seed=1)


@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (128, 32, 32), (129, 33, 33), (257, 70, 1000), (40, 300, 5)])
def test_f64tc_shapes(m, n, k):
    _check("N", "N", m, n, k, seed=m + n + k)


def test_f64tc_alpha_beta():
    _check("C", "N", 200, 150, 120, alpha=-1.0, beta=1.0, seed=3)
    _check("N", "C", 130, 64, 64, alpha=0.5 - 2j, beta=0.25 + 1j, seed=4)


def test_f64tc_row_range_and_split_k():
    # rows spread over 2^+-20 (row scales), and few output tiles with long K
    # (the K-split path)
    _check("N", "N", 96, 40, 3456, spread=20.0, seed=5)
    _check("C", "N", 128, 64, 6912, seed=6)


def test_f64tc_error_is_fp64_level():
    # on a well-scaled product the normwise error is that of an FP64 product
    err, scale = _check("N", "N", 512, 512, 512, seed=7)
    assert (err / scale).max() < 1.0
