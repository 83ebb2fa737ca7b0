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
