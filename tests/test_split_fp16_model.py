"""The number format of the mixed-precision contractions, checked on the CPU.

Each real row x of an operand is scaled by a power of two so that its largest
entry lies in [2^13, 2^14), rounded to FP32, and written as two FP16 values
hi = fp16(x), lo = fp16(x - hi) (x - hi is exact in FP32); a product keeps
hi_a hi_b + hi_a lo_b + lo_a hi_b.  numpy's float16 and float32 conversions
round to nearest even like the device conversions, so this model of the
format is exact; it shares no code with the kernels.  It pins:

* the two slices represent each scaled entry to 1.5 2^-9, i.e. 1.5 2^-22 of
  the row maximum ("~22 bits"), entries of any size included;
* dropping lo_a lo_b costs at most 2^-24 of the largest product;
* so a contraction of length K is within 4 K 2^-22 max|a| max|b| of the
  exact product before the FP32 accumulation; two BF16 slices keep 8 + 8
  significant bits of each entry (an error up to 2^-17 of it), which that
  bound does not allow.
"""
import math

import numpy as np


def scale_shift(row):
    mx = float(np.max(np.abs(row))) * 1.0000001
    if mx == 0.0:
        return 0
    _, e = math.frexp(mx)                  # mx in [2^(e-1), 2^e)
    return 14 - e                          # max 2^sh in [2^13, 2^14)


def split(row):
    sh = scale_shift(row)
    x = np.ldexp(row, sh).astype(np.float32)
    hi = x.astype(np.float16)
    lo = (x - hi.astype(np.float32)).astype(np.float16)
    return hi, lo, sh


def test_two_slices_hold_22_bits_of_the_row_maximum():
    rng = np.random.default_rng(0)
    for scale in (1.0, 1e-7, 3e5):
        # entries spread over twelve orders of magnitude below the maximum
        row = scale * rng.standard_normal(4096) * 10.0 ** rng.uniform(-12, 0, 4096)
        hi, lo, sh = split(row)
        assert np.all(np.isfinite(hi)) and np.all(np.isfinite(lo))
        rep = hi.astype(np.float64) + lo.astype(np.float64)
        err = np.abs(rep - np.ldexp(row, sh))
        assert err.max() <= 1.5 * 2.0 ** -9
        mx = np.abs(np.ldexp(row, sh)).max()
        assert 2.0 ** 13 <= mx < 2.0 ** 14
        assert err.max() / mx <= 1.5 * 2.0 ** -22
        # and the hi slice alone keeps only 11 bits
        assert np.abs(hi.astype(np.float64) - np.ldexp(row, sh)).max() / mx > 2.0 ** -16


def test_dropped_lo_lo_term_and_contraction_bound():
    rng = np.random.default_rng(1)
    K = 2048
    a = rng.standard_normal(K) * 10.0 ** rng.uniform(-3, 0, K)
    b = rng.standard_normal(K)
    ha, la, sa = split(a)
    hb, lb, sb = split(b)
    ha, la, hb, lb = (v.astype(np.float64) for v in (ha, la, hb, lb))
    # |lo| <= 4 in scaled units (half an FP16 ulp of values below 2^14)
    assert np.abs(la).max() <= 4 and np.abs(lb).max() <= 4
    assert np.abs(la * lb).max() <= 2.0 ** -24 * 2.0 ** 28
    # the kept pairs, summed exactly in FP64 (the FP32 accumulation is separate)
    kept = np.dot(ha, hb) + np.dot(ha, lb) + np.dot(la, hb)
    got = math.ldexp(kept, -(sa + sb))
    exact = float(np.dot(a, b))
    bound = 4 * K * 2.0 ** -22 * np.abs(a).max() * np.abs(b).max()
    assert abs(got - exact) <= bound
    # two unscaled BF16 slices (8 + 8 bits) would miss the same bound
    def bf16(v):
        u = np.asarray(v, np.float32).view(np.uint32).astype(np.uint64)
        u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
        return u.astype(np.uint32).view(np.float32).astype(np.float64)
    a1 = bf16(a)
    a2 = bf16(a - a1)
    b1 = bf16(b)
    b2 = bf16(b - b1)
    rep_err = max(np.abs(a1 + a2 - a).max() / np.abs(a).max(), np.abs(b1 + b2 - b).max() / np.abs(b).max())
    assert rep_err > 2.0 ** -22
