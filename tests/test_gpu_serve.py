"""pw_serve: continuous batching of fixed-potential eigensolves.  Each result
must be the same alone and in the mix; admission refuses what does not fit;
a bad request fails alone without disturbing the others."""
import numpy as np
import pytest

import synth
from oracle import pw_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _requests():
    reqs = synth.serving_requests(6, rate_per_s=20.0, seed=77)
    for r in reqs:                       # keep the GPU test small: 8-atom cells
        r["n"] = 1
        r["nbands"] = 18
    return reqs


def test_serve_alone_equals_mix_and_oracle():
    import paper_2406_10765_gb300 as pw
    reqs = _requests()
    mix = pw.pw_serve(reqs, max_slots=3, precision="fp64")
    for r, m in zip(reqs, mix):
        assert m["status"] == 0, m
        alone = pw.pw_serve([dict(r, t_arrival=0.0)], max_slots=1, precision="fp64")[0]
        assert np.array_equal(alone["eig"], m["eig"])
        assert m["max_resid"] <= 1e-8
    # the generated inputs are the seeded draws: dense diagonalisation agrees
    r, m = reqs[0], mix[0]
    ci = synth.cell_inputs(r["species"], 1, r["seed"])
    cell = O.make_cell(ci["L"], ci["tau"], ci["depth"], ci["dkb"], r["ecut"])
    w, _ = O.dense_eigs(cell, r["nbands"])
    assert np.abs(m["eig"] - w).max() < 1e-10
    assert all(x["latency"] >= 0 for x in mix)


def test_serve_mixed_precision_close_to_fp64():
    import paper_2406_10765_gb300 as pw
    reqs = _requests()[:3]
    a = pw.pw_serve(reqs, max_slots=3, precision="fp64")
    b = pw.pw_serve(reqs, max_slots=3, precision="mixed")
    for x, y in zip(a, b):
        assert x["status"] == 0 and y["status"] == 0
        assert np.abs(x["eig"] - y["eig"]).max() <= 1e-6
        assert y["orth_err"] <= 1e-10


def test_serve_admission_and_fault_isolation():
    import paper_2406_10765_gb300 as pw
    reqs = _requests()[:3]
    # nothing fits a 1 MB budget: every request is refused, none runs
    out = pw.pw_serve(reqs, max_slots=2, hbm_budget=1 << 20)
    assert all(o["status"] == pw.PW_ERR_BUSY for o in out)
    # an impossible band count fails on its own; the others are unaffected
    bad = dict(reqs[1], nbands=5000)
    out = pw.pw_serve([reqs[0], bad, reqs[2]], max_slots=3)
    assert out[0]["status"] == 0 and out[2]["status"] == 0
    assert out[1]["status"] == pw.PW_ERR_ARG


def test_serve_mixed_concurrent_equals_alone():
    # larger cells, all four slots busy: concurrency must not change a result
    import paper_2406_10765_gb300 as pw
    reqs = synth.serving_requests(2000, rate_per_s=50.0, seed=2024)[:6]
    for r in reqs:
        r["n"] = min(r["n"], 2)
        r["nbands"] = round(1.125 * 2 * 8 * r["n"] ** 3)
    mix = pw.pw_serve(reqs, max_slots=4, precision="mixed")
    for r, m in zip(reqs, mix):
        alone = pw.pw_serve([dict(r, t_arrival=0.0)], max_slots=1, precision="mixed")[0]
        assert m["status"] == alone["status"]
        assert np.array_equal(alone["eig"], m["eig"])
        assert m["status"] == 0 and m["max_resid"] <= 5e-6


def test_serve_autotuned_plans_within_tolerance():
    # with the autotuner on (FFT plan per grid size, K splits per shape class)
    # the served eigenvalues stay within the mixed-precision tolerance of the
    # untuned run, and every request still converges
    import paper_2406_10765_gb300 as pw
    reqs = synth.serving_requests(2000, rate_per_s=50.0, seed=2024)[:6]
    for r in reqs:
        r["n"] = min(r["n"], 2)
        r["nbands"] = round(1.125 * 2 * 8 * r["n"] ** 3)
    base = pw.pw_serve(reqs, max_slots=4, precision="mixed")
    try:
        pw.pw_autotune_gemm(1)
        tuned = pw.pw_serve(reqs, max_slots=4, precision="mixed", autotune=True)
    finally:
        pw.pw_autotune_gemm(0)
    for a, b in zip(base, tuned):
        assert a["status"] == 0 and b["status"] == 0, (a["status"], b["status"])
        assert np.abs(a["eig"] - b["eig"]).max() <= 2e-6
        assert b["max_resid"] <= 5e-6 and b["orth_err"] <= 1e-10


def test_serve_eight_slots_equals_alone():
    # eight requests of the seeded stream on eight slots at once (non-blocking
    # streams, many cells set up concurrently): each result bitwise equal to
    # the request served alone.  Cell tables and the divide-and-conquer tree
    # are uploaded in order on the request's stream; a plain pageable copy
    # may return before its DMA lands, and non-blocking streams do not wait
    # for it.
    import paper_2406_10765_gb300 as pw
    reqs = synth.serving_requests(2000, rate_per_s=1000.0, seed=2024)[:8]
    for r in reqs:
        r["n"] = min(r["n"], 2)
        r["nbands"] = round(1.125 * 2 * 8 * r["n"] ** 3)
    mix = pw.pw_serve(reqs, max_slots=8, precision="mixed")
    for r, m in zip(reqs, mix):
        assert m["status"] == 0, m["status"]
        alone = pw.pw_serve([dict(r, t_arrival=0.0)], max_slots=1, precision="mixed")[0]
        assert np.array_equal(alone["eig"], m["eig"])


def test_serve_cross_request_fft_batching():
    # six C-8 requests (all on the 16^3 grid, different Ecut: uneven spheres)
    # running at once: their FFT local parts share launches (one launch per
    # kernel carries several requests' band blocks), and every result is
    # bitwise the same as with each request launching its own kernels
    import paper_2406_10765_gb300 as pw
    reqs = [dict(species="C", n=1, ecut=8.0 + 0.7 * i, nbands=18, seed=100 + i, t_arrival=0.0)
            for i in range(6)]
    l0, j0 = pw.pw_fft_batch_stats()
    a = pw.pw_serve(reqs, max_slots=6, precision="mixed", batch_fft=True, batch_window_us=500.0)
    l1, j1 = pw.pw_fft_batch_stats()
    b = pw.pw_serve(reqs, max_slots=6, precision="mixed", batch_fft=False)
    assert pw.pw_fft_batch_stats() == (l1, j1)
    assert len({x["npw"] for x in a}) > 1
    for x, y in zip(a, b):
        assert x["status"] == 0 and y["status"] == 0
        assert np.array_equal(x["eig"], y["eig"])
    assert l1 > l0 and (j1 - j0) > (l1 - l0)       # some launches carried several requests
