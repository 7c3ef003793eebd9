"""The arithmetic claims behind the digit-sliced operator's tolerance, checked
on the CPU in exact arithmetic (Python integers and fractions), independent
of the CUDA code:

* eight signed 6-bit digits represent |v| <= 1 to within 2^-48, and every
  digit is an integer in [-32, 32] (exact in fp16): the kernel's form,
  balanced base-64 digits of the fixed-point integer rint(2^47 v), and the
  remainder form (first digit rint(2^5 v), then the remainder times 2^6,
  rounded) meet the same bound;
* a level sum D_c = sum over digit pairs s + t = c of the products over
  npts * nb terms stays below 2^24 in magnitude for c <= 5 at 81 x 48 terms
  (so FP32 holds it exactly), and the weighted recombination
  sum_{c<=8} D_c 2^(6 (8 - c)) + rint(D_9 2^-6) fits a signed 64-bit
  integer, up to nb = 64;
* keeping the levels c <= 9 (level 9 rounded to the unit of level 8)
  reproduces a dot product to within a small multiple of 2^-48 times the
  product of the two scales per term;
* the previous scheme (seven digits, levels c <= 8) is 2^6 times coarser, so
  the added digit and level are what bring the operator under 1e-12.
"""
from fractions import Fraction

import numpy as np
import pytest

BETA, TOP = 6, 5


def digits(v, n=8):
    """n digits of v (|v| <= 1) as Python ints, the remainder steps exact."""
    w = Fraction(v) * 2 ** TOP
    out = []
    for s in range(n):
        d = round(w)          # round half to even, like rint
        out.append(int(d))
        w = (w - d) * 2 ** BETA
    return out


def digits_int(v, n=8):
    """The kernel's digits: N = rint(v 2^(5 + 6 (n - 1))), then balanced
    base-64 digits from the bottom, d = ((N + 32) mod 64) - 32 and
    N <- (N - d) / 64, the remainder the top digit."""
    N = round(Fraction(v) * 2 ** (TOP + BETA * (n - 1)))    # ties to even, like rint
    out = []
    for _ in range(n - 1):
        d = (N + 32) % 64 - 32
        out.append(d)
        N = (N - d) // 64
    out.append(N)
    return out[::-1]


def value(ds):
    return sum(Fraction(d, 2 ** (TOP + BETA * s)) for s, d in enumerate(ds))


def rint_frac(q):
    """Round a Fraction to the nearest integer, ties to even (like rint)."""
    return round(q)


def test_representation_error_and_digit_range():
    rng = np.random.default_rng(5)
    vals = list(rng.uniform(-1, 1, 2000)) + [1.0, -1.0, 0.0, 2.0 ** -40, -0.5, 0.5 - 2 ** -53,
                                              1 - 2 ** -53, -(1 - 2 ** -53), 2 ** -48, 2 ** -49]
    for v in vals:
        for ds in (digits(v), digits_int(v)):
            assert len(ds) == 8
            assert all(-32 <= d <= 32 for d in ds), (v, ds)
            assert abs(value(ds) - Fraction(v)) <= Fraction(1, 2 ** 48), v
        # the kernel's low digits stay in [-32, 31]
        assert all(-32 <= d <= 31 for d in digits_int(v)[1:]), v


def test_level_sums_fit_fp32_and_int64():
    pmax = 32 * 32                    # largest digit product
    for K in (81 * 48, 81 * 64):      # terms per output element (bench shape, largest nb)
        for c in range(2, 10):
            bound = (c - 1) * K * pmax
            if c <= 4 or (c == 5 and K == 81 * 48):
                assert bound <= 2 ** 24   # exact in the FP32 accumulator
            # a level sum converts to int32 exactly (__float2int_rn)
            assert bound < 2 ** 31
        # recombination over the Re and Im input rows (four contributions to
        # each output), levels 2..8 shifted, level 9 divided by 2^6
        total = 2 * sum((c - 1) * K * pmax * 2 ** (BETA * (8 - c)) for c in range(2, 9))
        total += 2 * (8 * K * pmax // 2 ** 6 + 1)
        assert total < 2 ** 63


def dot_by_levels(a, x, ndig, maxlev, round9, split=None):
    split = split or (digits_int if ndig == 8 else digits)
    da = [split(v, ndig) for v in a]
    dx = [split(v, ndig) for v in x]
    D = {c: 0 for c in range(2, maxlev + 1)}
    for k in range(len(a)):
        for s in range(1, ndig + 1):
            for t in range(1, ndig + 1):
                if s + t <= maxlev:
                    D[s + t] += da[k][s - 1] * dx[k][t - 1]
    V = sum(D[c] * 2 ** (BETA * (8 - c)) for c in range(2, 9))
    if maxlev >= 9:
        V += rint_frac(Fraction(D[9], 2 ** BETA)) if round9 else Fraction(D[9], 2 ** BETA)
    return Fraction(V) / 2 ** (2 * TOP + 6 * BETA)     # 2^-46


@pytest.mark.parametrize("K", [16, 400])
def test_truncated_level_product_error(K):
    """sum_k a_k x_k from the digit pairs with s + t <= 9 and level 9 rounded
    to the unit of level 8, against the exact value: within 4 K 2^-48
    (representation of both operands, the dropped pairs s + t >= 10, each
    below 2^-48 per term, and half a unit 2^-46 for each rounding of level
    9 -- the kernel rounds the contributions of the Re and Im input rows
    separately, so up to 2^-46 per output)."""
    rng = np.random.default_rng(K)
    a = rng.uniform(-1, 1, K)
    x = rng.uniform(-1, 1, K)
    exact = sum(Fraction(u) * Fraction(v) for u, v in zip(a, x))
    approx = dot_by_levels(a, x, 8, 9, True)
    assert abs(approx - exact) <= Fraction(4 * K, 2 ** 48) + Fraction(1, 2 ** 46)
    # the remainder form of the digits meets the same bound
    alt = dot_by_levels(a, x, 8, 9, True, split=digits)
    assert abs(alt - exact) <= Fraction(4 * K, 2 ** 48) + Fraction(1, 2 ** 46)
    # the seven-digit scheme with levels <= 8 is bounded only at 2^-42
    old = dot_by_levels(a, x, 7, 8, False)
    assert abs(old - exact) <= Fraction(2 * K, 2 ** 42)


def test_dropped_level_is_a_real_term():
    """A plausible slip -- keeping only levels <= 8 with eight digits -- is
    caught: on inputs whose eighth digits are large the result moves by far
    more than the 2^-48 budget."""
    K = 64
    rng = np.random.default_rng(11)
    a = rng.uniform(-1, 1, K)
    x = rng.uniform(-1, 1, K)
    exact = sum(Fraction(u) * Fraction(v) for u, v in zip(a, x))
    full = dot_by_levels(a, x, 8, 9, True)
    short = dot_by_levels(a, x, 8, 8, True)
    assert abs(full - exact) < abs(short - exact) / 8
