"""pw_apply_H_noalloc: H psi for callers that cannot allocate device memory at
the call (their GPU memory is owned by their own allocator, or they cannot
take cudaMalloc's implicit synchronisation).  Its output must match
pw_apply_H on the same inputs, over two calls in a row that share the
library's static scratch array.  This file is collected last on purpose."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from gpu_util import cells, to_dev, rel  # noqa: E402


def _both(lib, x):
    import paper_2406_10765_gb300 as pw
    npw, nb = x.shape
    psi = to_dev(x)
    ref = pw.new_block(npw, nb)
    got = pw.new_block(npw, nb)
    got.fill_(float("nan"))
    pw.pw_apply_H(lib.h, psi, ref)
    pw.pw_apply_H_noalloc(lib.h, psi, got)
    torch.cuda.synchronize()
    return got.cpu().numpy(), ref.cpu().numpy()


def test_noalloc_matches_apply_h_twice():
    lib, orc, _ = cells("Si", 1, 10.0)
    for seed, nb in [(7, 24), (8, 9)]:          # two calls in a row, different sizes
        x = synth.draw_x0(seed, 8, orc.npw, nb)
        got, ref = _both(lib, x)
        assert np.all(np.isfinite(got))
        assert rel(got, ref) < 1e-12


def test_noalloc_matches_oracle():
    # the same operator as the oracle's H (FP64 parity bound of pw_apply_H)
    from oracle import pw_oracle as O
    lib, orc, _ = cells("C", 1, 8.0)
    x = synth.draw_x0(4, 8, orc.npw, 7)
    got, _ = _both(lib, x)
    assert rel(got, O.apply_H(orc, x)) < 1e-12


def test_noalloc_on_a_mixed_precision_cell_is_fp64():
    # a cell set to mixed precision still gets FP64 arithmetic from the
    # no-allocation entry point: it matches the FP64 operator, not the
    # split-precision one
    import paper_2406_10765_gb300 as pw
    from oracle import pw_oracle as O
    lib, orc, _ = cells("Si", 1, 10.0, precision="mixed")
    x = synth.draw_x0(6, 8, orc.npw, 5)
    psi = to_dev(x)
    got = pw.new_block(orc.npw, 5)
    for _ in range(2):
        pw.pw_apply_H_noalloc(lib.h, psi, got)
        torch.cuda.synchronize()
        assert rel(got.cpu().numpy(), O.apply_H(orc, x)) < 1e-12


def test_noalloc_atom_free_cell():
    # no atoms: no projectors, only the kinetic term (and a zero potential)
    import paper_2406_10765_gb300 as pw
    from oracle import pw_oracle as O
    ci = synth.cell_inputs("C", 1, 0)
    empty = np.zeros((0, 3)), np.zeros(0), np.zeros((0, 4))
    lib = pw.Cell(ci["L"], *empty, 8.0)
    orc = O.make_cell(ci["L"], *empty, 8.0)
    x = synth.draw_x0(2, 8, orc.npw, 3)
    for _ in range(2):
        got, ref = _both(lib, x)
        assert rel(got, ref) < 1e-12
        assert rel(got, O.apply_H(orc, x)) < 1e-12


def test_noalloc_full_size_cell():
    lib, orc, _ = cells("Si", 4, 10.0)
    x = synth.draw_x0(9, 512, orc.npw, 3)
    got, ref = _both(lib, x)
    assert rel(got, ref) < 1e-12


def test_noalloc_rejects_oversize():
    import paper_2406_10765_gb300 as pw
    lib, orc, _ = cells("Si", 4, 10.0)
    nb = 1152                                    # projector coefficients alone exceed the scratch
    psi = pw.new_block(lib.npw, nb)
    out = pw.new_block(lib.npw, nb)
    with pytest.raises(pw.PwError) as e:
        pw.pw_apply_H_noalloc(lib.h, psi, out)
    assert e.value.status == pw.PW_ERR_ARG
