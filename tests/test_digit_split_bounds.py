"""The arithmetic claims behind the digit-sliced operator's tolerance, checked
on the CPU in exact arithmetic (Python integers and fractions), independent
of the CUDA code:

* seven signed 6-bit digits (first digit from rint(2^5 v), then remainder
  times 2^6) represent |v| <= 1 to within 2^-42, and every digit is an
  integer in [-32, 32] (exact in fp16);
* a level sum D_c = sum over digit pairs s + t = c of the products over
  npts * nb terms stays below 2^24 in magnitude for c <= 5 at 81 x 48 terms
  (so FP32 holds it exactly), and the weighted recombination
  sum_c D_c 2^(6 (8 - c)) fits a signed 64-bit integer;
* keeping the levels c <= 8 reproduces a dot product to within a small
  multiple of 2^-42 times the product of the two scales per term.
"""
from fractions import Fraction

import numpy as np
import pytest

DIGITS, BETA, TOP = 7, 6, 5


def digits(v):
    """Digits of v (|v| <= 1) as Python ints, the remainder steps exact."""
    w = Fraction(v) * 2 ** TOP
    out = []
    for s in range(DIGITS):
        d = round(w)          # round half to even, like rint
        out.append(int(d))
        w = (w - d) * 2 ** BETA
    return out


def value(ds):
    return sum(Fraction(d, 2 ** (TOP + BETA * s)) for s, d in enumerate(ds))


def test_representation_error_and_digit_range():
    rng = np.random.default_rng(5)
    vals = list(rng.uniform(-1, 1, 2000)) + [1.0, -1.0, 0.0, 2.0 ** -40, -0.5, 0.5 - 2 ** -53]
    for v in vals:
        ds = digits(v)
        assert all(-32 <= d <= 32 for d in ds), (v, ds)
        assert abs(value(ds) - Fraction(v)) <= Fraction(1, 2 ** 42), v


def test_level_sums_fit_fp32_and_int64():
    K = 81 * 48                       # terms per output element at the bench shape
    pmax = 32 * 32                    # largest digit product
    for c in range(2, 9):
        pairs = c - 1
        bound = pairs * K * pmax
        if c <= 5:
            assert bound <= 2 ** 24   # exact in the FP32 accumulator
    # recombination: |sum_c D_c 2^(6(8-c))| over Re and Im input rows
    total = sum((c - 1) * K * pmax * 2 ** (BETA * (8 - c)) for c in range(2, 9)) * 2
    assert total < 2 ** 63
    # the largest basis size, nb = 64, keeps levels <= 4 exact
    K64 = 81 * 64
    assert 3 * K64 * pmax <= 2 ** 24


@pytest.mark.parametrize("K", [16, 400])
def test_truncated_level_product_error(K):
    """sum_k a_k x_k from the digit pairs with s + t <= 8, against the exact
    value: within 2 K 2^-42 (representation of both operands plus dropped
    pairs, each below 2^-42 per term)."""
    rng = np.random.default_rng(K)
    a = rng.uniform(-1, 1, K)
    x = rng.uniform(-1, 1, K)
    da = [digits(v) for v in a]
    dx = [digits(v) for v in x]
    D = {c: 0 for c in range(2, 9)}
    for k in range(K):
        for s in range(1, DIGITS + 1):
            for t in range(1, DIGITS + 1):
                if s + t <= 8:
                    D[s + t] += da[k][s - 1] * dx[k][t - 1]
    V = sum(D[c] * 2 ** (BETA * (8 - c)) for c in D)
    approx = Fraction(V, 2 ** (2 * TOP + 6 * BETA))     # 2^-46
    exact = sum(Fraction(u) * Fraction(v) for u, v in zip(a, x))
    assert abs(approx - exact) <= Fraction(2 * K, 2 ** 42)
