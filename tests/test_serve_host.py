"""Host-side pieces of the serving loop (no GPU): the admission footprint
model and the seeded request stream."""
import numpy as np

import synth


def test_footprint_model_monotone():
    import paper_2406_10765_gb300 as pw
    base = dict(species="Si", n=1, ecut=10.0, nbands=18, seed=0)
    f0 = pw.pw_request_footprint(base)
    assert f0 > 0
    assert pw.pw_request_footprint(dict(base, n=2)) > f0
    assert pw.pw_request_footprint(dict(base, ecut=12.0)) > f0
    assert pw.pw_request_footprint(dict(base, nbands=36)) > f0
    assert pw.pw_request_footprint(base, "mixed") > f0
    # Si-512 solve: tens of GB, below the 288 GB part
    big = pw.pw_request_footprint(dict(species="Si", n=4, ecut=10.0, nbands=1152, seed=0))
    assert 1e10 < big < 2e11


def test_footprint_counts_householder_slices():
    # a Rayleigh-Ritz order of 1,024 or more (3 x 342 bands) adds the digit
    # slices of the tensor-core Hermitian products: 9 tile rows, 45 lower
    # tiles of 512 KB, on top of what one more band costs
    import paper_2406_10765_gb300 as pw
    base = dict(species="Si", n=2, ecut=10.0, nbands=340, seed=0)
    f340, f341, f342 = (pw.pw_request_footprint(dict(base, nbands=b)) for b in (340, 341, 342))
    assert f342 - f341 > (f341 - f340) + 45 * 512 * 1024


def test_request_stream_shape():
    reqs = synth.serving_requests(2000, rate_per_s=5.0, seed=1)
    sp = np.array([r["species"] == "Si" for r in reqs])
    ns = np.array([r["n"] for r in reqs])
    ec = np.array([r["ecut"] for r in reqs])
    t = np.array([r["t_arrival"] for r in reqs])
    assert 0.45 < sp.mean() < 0.55
    assert set(ns) == {1, 2, 3}
    assert ec.min() >= 8.0 and ec.max() < 12.0
    assert np.all(np.diff(t) >= 0)
    gaps = np.diff(t)
    assert abs(gaps.mean() - 0.2) < 0.02            # Poisson rate 5/s
    assert all(r["nbands"] == round(1.125 * 2 * 8 * r["n"] ** 3) for r in reqs)
