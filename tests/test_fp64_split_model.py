"""The arithmetic of the FP64-accurate products on the FP16 tensor cores,
checked in exact integer arithmetic on the CPU.

A model of the scheme written from its definition (an Ozaki-type split):
each real row of A and each real column of B is scaled by a power of two so
that its largest entry lies in [1/2, 1); a scaled entry x is rounded to the
grid 2^-56 and written as sum_{p=1..8} d_p 2^(-7p) with integer digits; the
digit products with p + q = g (g = 2..9) are summed per chunk of 64 inner
indices (the FP32 tensor-memory accumulators), each group sum is added to a
64-bit fixed-point total at the binary point 2^-L, L = min(56, 62 -
ceil(log2 K)), and the total is converted to FP64 and unscaled.  It shares
no code with the kernels (which the GPU tests compare with the FP64
product); it pins the bounds the kernels rely on:

* the digits: |d_1| <= 2^7, |d_p| <= 2^6 after it (FP16 holds them
  exactly), and they reproduce the rounded entry exactly;
* every partial sum of a group over one chunk is an integer below 2^22, so
  an FP32 accumulator adds it exactly in any order;
* the pairs with p + q > 9 weigh less than 2^-55 of the largest product;
* the product's error per entry is at most 5.5 K 2^-55 max_k|a_ik| max_k|b_kj|
  (digit rounding 2^-57 of each scaled operand, the dropped pairs, the
  scales' factor of at most 4), plus the final rounding to FP64.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

S, BETA, CHUNK = 8, 7, 64


def scale_exp(v):
    """e with max|v| 2^e in [1/2, 1) (0 for an all-zero vector)."""
    mx = float(np.max(np.abs(v)))
    if mx == 0.0:
        return 0
    _, ex = math.frexp(mx)            # mx = f 2^ex, f in [1/2, 1)
    return -ex


def split(x, e):
    """Digits of round(x 2^(e + 56)) peeled from the top, 7 bits at a time,
    each rounded to nearest; the last digit takes the remainder."""
    F = round(Fraction(x) * 2 ** (e + 56))
    total = F
    d = []
    for p in range(1, S + 1):
        sh = 56 - BETA * p
        if sh > 0:
            q = (F + (1 << (sh - 1))) >> sh
            F -= q << sh
        else:
            q, F = F, 0
        d.append(q)
    return d, total


def shifted(v, sh):
    return v << sh if sh >= 0 else (v + (1 << (-sh - 1))) >> (-sh)


def model_product(A, B):
    """C = A B (real) through the split scheme; returns C and the largest
    group partial sum seen in any chunk."""
    m, K = A.shape
    n = B.shape[1]
    ea = [scale_exp(A[i]) for i in range(m)]
    eb = [scale_exp(B[:, j]) for j in range(n)]
    DA = np.zeros((S, m, K), dtype=np.int64)
    DB = np.zeros((S, K, n), dtype=np.int64)
    for i in range(m):
        for k in range(K):
            DA[:, i, k] = split(float(A[i, k]), ea[i])[0]
    for j in range(n):
        for k in range(K):
            DB[:, k, j] = split(float(B[k, j]), eb[j])[0]
    lg = max(0, math.ceil(math.log2(max(1, K))))
    L = min(56, 62 - lg)
    acc = [[0] * n for _ in range(m)]
    peak = 0
    for c0 in range(0, K, CHUNK):
        c1 = min(K, c0 + CHUNK)
        for g in range(2, S + 2):
            Sg = np.zeros((m, n), dtype=np.int64)
            for p in range(1, g):
                q = g - p
                if q > S:
                    continue
                Sg += DA[p - 1][:, c0:c1] @ DB[q - 1][c0:c1]
            # every prefix of the chunk's sum is bounded by the sum of |terms|
            absum = sum(np.abs(DA[p - 1][:, c0:c1]) @ np.abs(DB[g - p - 1][c0:c1])
                        for p in range(1, g) if g - p <= S)
            peak = max(peak, int(absum.max()))
            for i in range(m):
                for j in range(n):
                    acc[i][j] += shifted(int(Sg[i, j]), L - BETA * g)
    C = np.empty((m, n))
    for i in range(m):
        for j in range(n):
            assert abs(acc[i][j]) < 2 ** 63
            C[i, j] = math.ldexp(float(acc[i][j]), -L - ea[i] - eb[j])
    return C, peak


def exact_product(A, B):
    m, K = A.shape
    n = B.shape[1]
    return [[sum(Fraction(float(A[i, k])) * Fraction(float(B[k, j])) for k in range(K))
             for j in range(n)] for i in range(m)]


def test_digit_bounds_and_exact_reconstruction():
    rng = np.random.default_rng(0)
    xs = np.concatenate([rng.uniform(-1, 1, 2000), [0.999999999999, -0.9999999999999999, 0.5, -0.5,
                                                    1e-300, 2.0 ** -60, 0.0]])
    for x in xs:
        d, F = split(float(x), 0)
        assert abs(d[0]) <= 2 ** BETA and all(abs(v) <= 2 ** (BETA - 1) for v in d[1:])
        assert sum(v << (56 - BETA * (p + 1)) for p, v in enumerate(d)) == F
        # the rounded entry is within 2^-57 of x
        assert abs(Fraction(F, 2 ** 56) - Fraction(float(x))) <= Fraction(1, 2 ** 57)
        # FP16 holds every digit exactly (integers up to 2^11)
        assert all(float(np.float16(v)) == v for v in d)


def test_group_sums_fit_an_fp32_accumulator():
    # worst case over one chunk: every digit at its bound
    top = [2 ** BETA] + [2 ** (BETA - 1)] * (S - 1)
    for g in range(2, S + 2):
        worst = CHUNK * sum(top[p - 1] * top[g - p - 1] for p in range(1, g) if g - p <= S)
        assert worst < 2 ** 22 < 2 ** 24
    # the dropped pairs: p + q >= 10, relative to a largest product of 1
    dropped = sum(top[p - 1] * top[q - 1] * 2.0 ** (-BETA * (p + q))
                  for p in range(1, S + 1) for q in range(1, S + 1) if p + q > S + 1)
    assert dropped < 2.0 ** -55


KINDS = ["uniform", "rows_graded", "cols_graded", "sparse_large", "ragged"]


@pytest.mark.parametrize("kind", KINDS)
def test_model_product_error_bound(kind):
    rng = np.random.default_rng(KINDS.index(kind))
    m, n, K = 5, 4, 200
    A = rng.standard_normal((m, K))
    B = rng.standard_normal((K, n))
    if kind == "rows_graded":
        A *= np.logspace(-6, 6, m)[:, None]
        B *= np.logspace(3, -3, n)[None, :]
    elif kind == "cols_graded":
        A *= np.logspace(-3, 3, K)[None, :]             # wide range inside each row
    elif kind == "sparse_large":
        A[:, ::17] *= 1e8
        B[::13] *= 1e-5
    elif kind == "ragged":
        K = 130                                          # two full chunks and a tail of 2
        A, B = A[:, :K], B[:K]
    C, peak = model_product(A, B)
    assert peak < 2 ** 22
    ref = exact_product(A, B)
    for i in range(m):
        for j in range(n):
            bound = 5.5 * K * 2.0 ** -55 * np.abs(A[i]).max() * np.abs(B[:, j]).max()
            err = abs(Fraction(float(C[i, j])) - ref[i][j])
            assert err <= Fraction(bound) + abs(ref[i][j]) * Fraction(1, 2 ** 53), (i, j)


def test_model_product_beats_the_fp64_bound_on_uniform_rows():
    # rows without internal range: the split product's bound (5.5 K 2^-55
    # max|a| max|b|) is below the FP64 product's K u sum|a||b| (u = 2^-53)
    rng = np.random.default_rng(1)
    A = rng.uniform(0.5, 1.0, (3, 256))
    B = rng.uniform(0.5, 1.0, (256, 3))
    K = 256
    for i in range(3):
        for j in range(3):
            split_bound = 5.5 * K * 2.0 ** -55 * A[i].max() * B[:, j].max()
            fp64_bound = K * 2.0 ** -53 * float(np.abs(A[i]) @ np.abs(B[:, j]))
            assert split_bound < fp64_bound
    C, _ = model_product(A, B)
    ref = exact_product(A, B)
    assert max(abs(Fraction(float(C[i, j])) - ref[i][j]) / abs(ref[i][j])
               for i in range(3) for j in range(3)) < 2 ** -50
