"""FP64 GPU Hermitian eigensolver (the small dense eigensolve of the
Rayleigh-Ritz step, Syevd in Sec. III-D) against LAPACK."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _herm(n, seed, kind="rand"):
    rng = np.random.default_rng(seed)
    if kind == "rand":
        M = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
        return M + M.conj().T
    if kind == "degenerate":    # eigenvalues with multiplicity, random unitary
        w = np.repeat(np.arange(n // 4 + 1, dtype=float), 4)[:n]
        Q, _ = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
        return (Q * w) @ Q.conj().T
    if kind == "diag":
        return np.diag(rng.standard_normal(n)).astype(complex)
    if kind == "cluster":
        w = np.sort(np.concatenate([np.full(n // 2, 1.0) + 1e-12 * rng.standard_normal(n // 2),
                                    rng.standard_normal(n - n // 2)]))
        Q, _ = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
        return (Q * w) @ Q.conj().T
    raise ValueError(kind)


@pytest.mark.parametrize("n,nb,kind", [(1, 1, "rand"), (2, 1, "rand"), (3, 3, "rand"),
                                       (33, 11, "rand"), (72, 24, "rand"), (130, 40, "degenerate"),
                                       (97, 30, "diag"), (200, 64, "cluster"), (515, 170, "rand")])
def test_heev_matches_lapack(n, nb, kind):
    import paper_2406_10765_gb300 as pw
    A = _herm(n, n + 7, kind)
    w, Y = pw.pw_heev(torch.from_numpy(A).cuda(), nb)
    torch.cuda.synchronize()
    w = w.cpu().numpy()
    Y = Y.cpu().numpy()
    ref = np.linalg.eigvalsh(A)
    scale = max(1.0, np.abs(ref).max())
    assert np.abs(w - ref).max() < 1e-13 * scale * max(1, n) ** 0.5
    # eigenvectors: residual and orthonormality (unique only up to degenerate subspaces)
    assert np.abs(A @ Y - Y * w[:nb]).max() < 1e-12 * scale
    assert np.abs(Y.conj().T @ Y - np.eye(nb)).max() < 1e-12


def test_heev_argument_errors():
    from paper_2406_10765_gb300 import binding as B
    st = B._stream(None)
    import ctypes as ct
    assert B._heev(0, 1, ct.c_void_p(1), ct.c_void_p(1), ct.c_void_p(1), st) == B.PW_ERR_ARG
    assert B._heev(4, 5, ct.c_void_p(1), ct.c_void_p(1), ct.c_void_p(1), st) == B.PW_ERR_ARG


@pytest.mark.parametrize("mode,panels", [(0, 0), (1, 0), (1, 1), (1, 2), (1, 3)])
def test_heev_large_both_product_modes(mode, panels):
    # order 1,700: the panel updates, back-transformation and their K-split
    # products run on the FP64-accurate tensor-core path (mode 1) or the FP64
    # pipe (mode 0); the Householder columns as chained kernels with the
    # Hermitian products of the large panels on the tensor cores (panels 0,
    # mode 1), one cooperative launch per panel (panels 1), chained kernels
    # with every Hermitian product on the FP64 pipe (panels 2) or one
    # cooperative launch per large panel with its products on the tensor
    # cores (panels 3); all match LAPACK at the same tolerances
    import paper_2406_10765_gb300 as pw
    n, nb = 1700, 600
    A = _herm(n, 17, "rand")
    pw.pw_dense_products(mode)
    pw.pw_householder_panels(panels)
    try:
        w, Y = pw.pw_heev(torch.from_numpy(A).cuda(), nb)
        torch.cuda.synchronize()
    finally:
        pw.pw_dense_products(1)
        pw.pw_householder_panels(0)
    w = w.cpu().numpy()
    Y = Y.cpu().numpy()
    ref = np.linalg.eigvalsh(A)
    scale = max(1.0, np.abs(ref).max())
    assert np.abs(w - ref).max() < 1e-13 * scale * n ** 0.5
    assert np.abs(A @ Y - Y * w[:nb]).max() < 1e-12 * scale
    assert np.abs(Y.conj().T @ Y - np.eye(nb)).max() < 1e-12


def test_heev_cooperative_panels_match_chained():
    # the cooperative panel kernel runs the FP64-pipe chained kernels'
    # arithmetic in the same order (the compiler may contract multiply-adds
    # differently in the two kernels, so the last bits can differ):
    # eigenvalues to rounding and the same wanted subspace, on small and
    # ragged orders
    import paper_2406_10765_gb300 as pw
    for n, nb in [(2, 1), (33, 11), (130, 40), (515, 170)]:
        A = _herm(n, n + 3, "rand")
        out = []
        for coop in (2, 1):
            pw.pw_householder_panels(coop)
            try:
                w, Y = pw.pw_heev(torch.from_numpy(A).cuda(), nb)
                torch.cuda.synchronize()
                out.append((w.cpu().numpy(), Y.cpu().numpy()))
            finally:
                pw.pw_householder_panels(0)
        scale = max(1.0, np.abs(out[0][0]).max())
        assert np.abs(out[0][0] - out[1][0]).max() < 1e-13 * scale * n ** 0.5, n
        Ya, Yb = out[0][1], out[1][1]
        assert np.abs(Ya @ Ya.conj().T - Yb @ Yb.conj().T).max() < 1e-10, n
        assert np.abs(A @ Yb - Yb * out[1][0][:nb]).max() < 1e-12 * scale, n


@pytest.mark.parametrize("n,nb,kind", [(1025, 341, "rand"), (1100, 300, "degenerate"), (1200, 333, "cluster"),
                                       (1301, 420, "rand"), (1150, 250, "range")])
def test_heev_tensor_hermitian_products_match_fp64(n, nb, kind):
    # the Hermitian products of the panels with trailing order >= 1024 on the
    # tensor cores (slices of the trailing matrix) against the same chain on
    # the FP64 pipe, and both against LAPACK: ragged orders (partial 128-row
    # tiles, a panel boundary inside a tile), degenerate and clustered
    # spectra, and a matrix whose entries span six orders of magnitude (one
    # scale for the whole trailing matrix: the error is normwise; the FP64
    # products on the tensor cores are accurate relative to row and column
    # maxima, so much wider ranges lose digits against LAPACK in either mode)
    import paper_2406_10765_gb300 as pw
    if kind == "range":
        rng = np.random.default_rng(n)
        d = 10.0 ** rng.uniform(-3, 3, n)
        M = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
        A = (M + M.conj().T) * np.sqrt(np.outer(d, d)) * 1e-6 + np.diag(d)
    else:
        A = _herm(n, n + 5, kind)
    ref = np.linalg.eigvalsh(A)
    scale = max(1.0, np.abs(ref).max())
    out = []
    for panels in (0, 2, 3):
        pw.pw_householder_panels(panels)
        try:
            w, Y = pw.pw_heev(torch.from_numpy(A).cuda(), nb)
            torch.cuda.synchronize()
        finally:
            pw.pw_householder_panels(0)
        w, Y = w.cpu().numpy(), Y.cpu().numpy()
        assert np.abs(w - ref).max() < 1e-13 * scale * n ** 0.5, (panels, np.abs(w - ref).max() / scale)
        assert np.abs(A @ Y - Y * w[:nb]).max() < 1e-12 * scale, panels
        assert np.abs(Y.conj().T @ Y - np.eye(nb)).max() < 1e-12, panels
        out.append((w, Y))
    for k in (1, 2):
        assert np.abs(out[0][0] - out[k][0]).max() < 1e-13 * scale * n ** 0.5
    if kind == "rand":
        # a gap after the wanted pairs: the same wanted subspace
        Ya = out[0][1]
        for k in (1, 2):
            Yb = out[k][1]
            assert np.abs(Ya @ Ya.conj().T - Yb @ Yb.conj().T).max() < 1e-9
