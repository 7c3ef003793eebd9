"""Pins of the quantised operators evaluated by the low-precision GPU paths:
power-of-two scales, round-to-nearest-even codes checked against the IEEE
bit-level rule, and the error of the quantised operator against FP64."""
import numpy as np

from oracle.lowprec import (column_scales, lowprec_apply, pow2_scale, quantise_op, quantise_vec,
                            remainder, round_real, site_diagonal, site_scales)
from oracle.ops import coarse_op_apply
from synth import coarse_op, stencil, vectors


def test_pow2_scale(rng):
    m = np.abs(rng.standard_normal(1000)) * 10.0 ** rng.integers(-20, 20, 1000)
    s = pow2_scale(m)
    assert np.all((s / 2 < m) & (m <= s))
    assert np.all(np.log2(s) == np.round(np.log2(s)))
    e = np.arange(-30, 30)
    assert np.array_equal(pow2_scale(2.0 ** e), 2.0 ** e)
    assert pow2_scale(0.0) == 1.0


def _bf16_rne_bits(x32):
    """Round float32 to bfloat16 by the IEEE round-to-nearest-even rule on the
    bit pattern: add 0x7fff + lsb of the kept half, truncate 16 bits."""
    u = x32.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def test_bf16_rounding_matches_bit_rule(rng):
    x = rng.standard_normal(100000) * 10.0 ** rng.integers(-5, 5, 100000)
    x32 = x.astype(np.float32)
    assert np.array_equal(round_real(x, "bf16"), _bf16_rne_bits(x32))
    # ties go to even
    t = np.array([1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8], dtype=np.float32)
    assert np.array_equal(round_real(t, "bf16"), [1.0, 1.0 + 4 * 2.0 ** -8])


def test_fp16_rounding(rng):
    x = rng.uniform(-1, 1, 100000)
    q = round_real(x, "fp16")
    assert np.array_equal(q, x.astype(np.float32).astype(np.float16).astype(np.float64))
    assert np.max(np.abs(q - x)) <= 2.0 ** -12 + 2.0 ** -24   # half ulp at [0.5, 1) plus the FP32 step


def test_quantised_operator_error():
    L, nb, npts, R = (3, 2, 2, 3), 8, 81, 4
    disp, _ = stencil(npts)
    A = coarse_op(L, nb, npts, 17, 6.0)
    X = vectors(L, nb, R, 17)
    s = site_scales(A)
    d = site_diagonal(A)
    assert np.all(np.abs(d - 6.0) < 1.0)            # the shift sits on the diagonal
    Ar = remainder(A)
    assert np.allclose(Ar[:, 1:], A[:, 1:]) and np.allclose(
        np.real(np.trace(Ar[:, 0], axis1=-2, axis2=-1)), 0, atol=1e-5)
    ma = np.maximum(np.abs(Ar.real), np.abs(Ar.imag)).reshape(A.shape[0], -1).max(1)
    assert np.all((s / 2 < ma) & (ma <= s))
    sig = column_scales(X)
    assert sig.shape == (R,)
    Y = coarse_op_apply(A, X, L, disp)
    for kind, bits in (("fp32", 24), ("bf16", 8), ("fp16", 11)):
        Aq = quantise_op(A, kind)
        Xq = quantise_vec(X, kind)
        if kind != "fp32":
            codes = (quantise_op(A, kind) - A)[:, 1:] / s[:, None, None, None]
            assert np.max(np.abs(codes)) <= 2.0 ** -bits * np.sqrt(2)
            # the diagonal shift is carried exactly: error relative to the remainder scale
            rel_a = np.max(np.abs(Aq - A) / s[:, None, None, None])
            assert rel_a <= 2.0 ** -bits * np.sqrt(2) * 1.0001
        else:
            rel = np.max(np.abs(Aq - A) / np.maximum(np.abs(A), 1e-300))
            assert rel <= 2.0 ** -24 * np.sqrt(2)
        Yq = lowprec_apply(A, X, L, disp, kind)
        err = np.linalg.norm(Yq - Y) / np.linalg.norm(Y)
        assert err <= 2.0 ** -(bits - 4)
        if kind == "fp32":
            assert np.allclose(Yq, coarse_op_apply(Aq, Xq, L, disp))


def test_split16_two_terms(rng):
    from oracle.lowprec import split16
    u = rng.uniform(-1, 1, 100000) * 10.0 ** rng.integers(-3, 1, 100000)
    u32 = u.astype(np.float32).astype(np.float64)
    hi, lo = split16(u)
    assert np.array_equal(hi, u32.astype(np.float16).astype(np.float64))
    rel = np.abs(hi + 2.0 ** -11 * lo - u32) / np.abs(u32)
    assert np.max(rel[np.abs(u32) > 2.0 ** -10]) <= 2.0 ** -21


def test_split_operators_accuracy():
    """fp16x is linear in X to ~2^-22 (its error is the fp16 coefficients');
    tc32 reaches FP32-class accuracy."""
    L, nb, npts, R = (3, 2, 2, 3), 8, 81, 4
    disp, _ = stencil(npts)
    A = coarse_op(L, nb, npts, 23, 9.0)
    X = vectors(L, nb, R, 23)
    Y = coarse_op_apply(A, X, L, disp)
    e16 = np.linalg.norm(lowprec_apply(A, X, L, disp, "fp16") - Y) / np.linalg.norm(Y)
    e16x = np.linalg.norm(lowprec_apply(A, X, L, disp, "fp16x") - Y) / np.linalg.norm(Y)
    e32 = np.linalg.norm(lowprec_apply(A, X, L, disp, "tc32") - Y) / np.linalg.norm(Y)
    assert e16x <= e16 and e16x <= 2.0 ** -9
    assert e32 <= 2.0 ** -19
    # linearity in X: fp16x(a X1 + X2) vs a fp16x(X1) + fp16x(X2)
    X2 = vectors(L, nb, R, 24)
    lhs = lowprec_apply(A, 0.37 * X + X2, L, disp, "fp16x")
    rhs = 0.37 * lowprec_apply(A, X, L, disp, "fp16x") + lowprec_apply(A, X2, L, disp, "fp16x")
    lin16 = np.linalg.norm(lowprec_apply(A, 0.37 * X + X2, L, disp, "fp16")
                           - 0.37 * lowprec_apply(A, X, L, disp, "fp16")
                           - lowprec_apply(A, X2, L, disp, "fp16")) / np.linalg.norm(rhs)
    assert np.linalg.norm(lhs - rhs) / np.linalg.norm(rhs) <= 2.0 ** -19 < lin16
