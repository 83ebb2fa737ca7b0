"""Split-FP16 tcgen05 GEMM (mixed-precision contractions) against an FP64
reference product of the same operands."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _cm(x):
    """host complex -> column-major CUDA tensor"""
    return torch.from_numpy(np.ascontiguousarray(x.T)).cuda().T


def _rand(shape, seed, scale=1.0):
    rng = np.random.default_rng(seed)
    return scale * (rng.standard_normal(shape) + 1j * rng.standard_normal(shape))


@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (64, 256, 512), (100, 37, 1000), (300, 300, 2000)])
def test_tc_gemm_AhB(m, n, k):
    import paper_2406_10765_gb300 as pw
    A = _rand((k, m), 1, 1e-2)
    B = _rand((k, n), 2, 3.0)
    C = pw.pw_zgemm_tc("C", _cm(A), _cm(B)).cpu().numpy()
    ref = A.conj().T @ B
    bound = np.sqrt(k) * np.abs(A).max() * np.abs(B).max()
    assert np.abs(C - ref).max() < 2e-6 * bound


@pytest.mark.parametrize("m,n,k", [(129, 5, 40), (1000, 64, 300), (257, 130, 1200)])
def test_tc_gemm_AB_accumulate(m, n, k):
    import paper_2406_10765_gb300 as pw
    A = _rand((m, k), 3, 0.5)
    B = _rand((k, n), 4, 2.0)
    C0 = _rand((m, n), 5)
    C = pw.pw_zgemm_tc("N", _cm(A), _cm(B), C=_cm(C0).clone(), beta=1.0).cpu().numpy()
    ref = C0 + A @ B
    bound = np.sqrt(k) * np.abs(A).max() * np.abs(B).max()
    assert np.abs(C - ref).max() < 2e-6 * bound


def test_tc_gemm_gram_hermitian():
    import paper_2406_10765_gb300 as pw
    S = _rand((5000, 200), 6, 0.01)
    G = pw.pw_zgemm_tc("C", _cm(S), _cm(S)).cpu().numpy()
    ref = S.conj().T @ S
    assert np.abs(G - ref).max() < 1e-6 * np.abs(ref).max()


@pytest.mark.parametrize("split", [2, 3, 4])
def test_tc_gemm_k_split(split):
    # K cut into `split` parts per tile, FP64 partial sums reduced in order:
    # A^H B, the Hermitian Gram and A B + C agree with the FP64 products
    import paper_2406_10765_gb300 as pw
    try:
        pw.pw_autotune_gemm(2, split)
        A = _rand((3000, 100), 11, 1e-2)
        B = _rand((3000, 37), 12, 3.0)
        C = pw.pw_zgemm_tc("C", _cm(A), _cm(B)).cpu().numpy()
        bound = np.sqrt(3000) * np.abs(A).max() * np.abs(B).max()
        assert np.abs(C - A.conj().T @ B).max() < 2e-6 * bound
        S = _rand((5000, 200), 6, 0.01)
        G = pw.pw_zgemm_tc("C", _cm(S), _cm(S)).cpu().numpy()
        ref = S.conj().T @ S
        assert np.abs(G - ref).max() < 1e-6 * np.abs(ref).max()
        A2 = _rand((257, 1200), 3, 0.5)
        B2 = _rand((1200, 130), 4, 2.0)
        C0 = _rand((257, 130), 5)
        C2 = pw.pw_zgemm_tc("N", _cm(A2), _cm(B2), C=_cm(C0).clone(), beta=1.0).cpu().numpy()
        bound = np.sqrt(1200) * np.abs(A2).max() * np.abs(B2).max()
        assert np.abs(C2 - (C0 + A2 @ B2)).max() < 2e-6 * bound
    finally:
        pw.pw_autotune_gemm(0)


def test_tc_gemm_autotuned_split():
    # mode 1: the first call of each few-tile shape times the candidate
    # splits and records the fastest; results stay within the same bound
    import paper_2406_10765_gb300 as pw
    try:
        pw.pw_autotune_gemm(1)
        A = _rand((20000, 256), 21, 1e-2)
        B = _rand((20000, 128), 22, 1.0)
        for _ in range(2):
            C = pw.pw_zgemm_tc("C", _cm(A), _cm(B)).cpu().numpy()
            bound = np.sqrt(20000) * np.abs(A).max() * np.abs(B).max()
            assert np.abs(C - A.conj().T @ B).max() < 2e-6 * bound
        table = pw.pw_autotune_gemm_table()
        lines = [ln for ln in table.splitlines() if ln]
        assert len(lines) >= 1
        split = int(lines[0].split("split=")[1].split()[0])
        assert split >= 1
    finally:
        pw.pw_autotune_gemm(0)
    assert pw.pw_autotune_gemm_table() == ""


def test_bounded_wait_reports_and_context_survives():
    # the pipeline's bounded wait on a barrier nothing arrives on gives up
    # after the limit and reports (no fault, no hang); the context stays
    # usable for the next product
    import paper_2406_10765_gb300 as pw
    assert pw.pw_selftest_bounded_wait(2_000_000) == pw.PW_ERR_TIMEOUT
    assert pw.pw_selftest_bounded_wait(0) == pw.PW_ERR_ARG
    A = _rand((500, 40), 31, 0.1)
    B = _rand((500, 30), 32, 1.0)
    C = pw.pw_zgemm_tc("C", _cm(A), _cm(B)).cpu().numpy()
    bound = np.sqrt(500) * np.abs(A).max() * np.abs(B).max()
    assert np.abs(C - A.conj().T @ B).max() < 2e-6 * bound
