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
