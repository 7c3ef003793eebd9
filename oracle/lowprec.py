"""Quantised operators evaluated by the low-precision GPU paths.

Test infrastructure only (see the package docstring).

The paper runs in FP64 and notes that the multigrid preconditioner tolerates
single precision (Sec. 4, conclusions); the reduced-precision forms here are
this library's own.  Each is defined so that the GPU evaluates it exactly up
to the order of its FP32 accumulation:

* FP32 operator: coefficients and vectors rounded to complex64.
* BF16 / FP16 operator: the mean real diagonal of the self block,
  d_x = (1/nb) sum_a Re A_0(x)_aa, is rounded to FP32 and kept out of the
  quantisation (a large shift c I would otherwise cost a rounding error of
  c 2^-9 on every diagonal entry, far above the smallest eigenvalue).  The
  remaining block A'(x) = [A_0(x) - d_x I, A_1(x), ..., A_{Np-1}(x)] is
  divided by a power of two s_x = 2^e, e the least integer with
  max |Re|, |Im| <= 2^e (so the scaled entries lie in [-1, 1]), and rounded
  FP64 -> FP32 -> BF16/FP16, round-to-nearest-even at each step.  Each
  right-hand side column r of the complex64 input is divided by its own power
  of two sigma_r (same rule over the whole column) and rounded to BF16/FP16.
  The result is
      Y(x) = s_x sigma_r sum_p Ahat_p(x) Xhat(x + delta_p) + d_x X(x).
Both roundings use the same two-step path on both sides, so the quantised
codes are bit-identical.

Two-term (split) forms, for the tensor-core paths that need FP32-class
accuracy from 16-bit operands (up to 32 right-hand sides):
* a value u (an FP32 number) is held as hi = fp16(u) and
  lo = fp16((u - hi) * 2^11), u ~ hi + 2^-11 lo to about 2^-22 relative;
* "fp16x": FP16 coefficient codes as above, input columns in two terms:
      Y = s_x sigma_r sum_p Ahat_p (Xhi + 2^-11 Xlo) + d_x X(x);
* "tc32": coefficients and input in two terms, the lo x lo product dropped:
      Y = s_x sigma_r sum_p [Ahi (Xhi + 2^-11 Xlo) + 2^-11 Alo Xhi] + d_x X(x).
"""
import numpy as np
import torch


def pow2_scale(m):
    """2^e with e the least integer such that m <= 2^e (m >= 0); 1 for m == 0."""
    m = np.asarray(m, dtype=np.float64)
    f, e = np.frexp(m)                      # m = f 2^e, f in [0.5, 1)
    e = np.where(f == 0.5, e - 1, e)
    return np.where(m > 0, np.ldexp(1.0, e), 1.0)


def round_real(x, kind):
    """FP64 -> FP32 (RN) -> kind (RN); returns the rounded values as float64."""
    x32 = np.asarray(x, dtype=np.float64).astype(np.float32)
    if kind == "fp32":
        return x32.astype(np.float64)
    t = torch.from_numpy(np.ascontiguousarray(x32))
    dt = torch.bfloat16 if kind == "bf16" else torch.float16
    return t.to(dt).to(torch.float64).numpy()


def round_complex(z, kind):
    return round_real(np.real(z), kind) + 1j * round_real(np.imag(z), kind)


def site_diagonal(A):
    """d_x: mean real diagonal of the self block, rounded to FP32."""
    nb = A.shape[2]
    d = np.real(np.trace(A[:, 0], axis1=-2, axis2=-1)) / nb
    return d.astype(np.float32).astype(np.float64)


def remainder(A):
    """A with d_x I taken off the self block."""
    Ar = A.astype(np.complex128).copy()
    Ar[:, 0] -= site_diagonal(A)[:, None, None] * np.eye(A.shape[2])[None]
    return Ar


def site_scales(A):
    """s_x for the remainder block of coefficients A[x][p][a][b]."""
    Ar = remainder(A)
    m = np.maximum(np.abs(Ar.real), np.abs(Ar.imag)).reshape(A.shape[0], -1).max(axis=1)
    return pow2_scale(m)


def column_scales(X):
    """sigma_r for vectors X[x][b][r]."""
    m = np.maximum(np.abs(X.real), np.abs(X.imag)).reshape(-1, X.shape[-1]).max(axis=0)
    return pow2_scale(m)


def quantise_op(A, kind):
    """Dequantised coefficients s_x * Ahat(x) that the GPU multiplies with."""
    if kind == "fp64":
        return A.astype(np.complex128)
    if kind == "fp32":
        return round_complex(A, "fp32")
    s = site_scales(A)
    q = round_complex(remainder(A) / s[:, None, None, None], kind) * s[:, None, None, None]
    q[:, 0] += site_diagonal(A)[:, None, None] * np.eye(A.shape[2])[None]
    return q


def quantise_vec(X, kind):
    """Dequantised input vectors sigma_r * Xhat.  X is taken as complex64
    input (the low-precision operators read FP32 vectors).  The d_x X(x)
    term of a BF16/FP16 application uses X in complex64, unquantised: see
    ``lowprec_apply``."""
    if kind == "fp64":
        return X.astype(np.complex128)
    X32 = round_complex(X, "fp32")
    if kind == "fp32":
        return X32
    sig = column_scales(X32)
    return round_complex(X32 / sig, kind) * sig


def split16(u):
    """(hi, lo) of FP32 values u: hi = fp16(u), lo = fp16((u - hi) * 2^11)."""
    u32 = np.asarray(u, dtype=np.float64).astype(np.float32)
    hi = u32.astype(np.float16).astype(np.float32)
    lo = ((u32 - hi) * np.float32(2048.0)).astype(np.float16).astype(np.float32)
    return hi.astype(np.float64), lo.astype(np.float64)


def split16_complex(z):
    hr, lr = split16(np.real(z))
    hi_, li = split16(np.imag(z))
    return hr + 1j * hi_, lr + 1j * li


def lowprec_apply(A, X, L, disp, kind):
    """The exact value the GPU operator of precision `kind` approximates with
    FP32 accumulation (FP64 arithmetic on the quantised operands)."""
    from .ops import coarse_op_apply
    if kind in ("fp64", "fp32"):
        return coarse_op_apply(quantise_op(A, kind), quantise_vec(X, kind), L, disp)
    if kind in ("fp16x", "tc32"):
        s = site_scales(A)
        u = remainder(A) / s[:, None, None, None]
        X32 = round_complex(X, "fp32")
        sig = column_scales(X32)
        xh, xl = split16_complex(X32 / sig)
        xh, xl = xh * sig, xl * sig
        if kind == "fp16x":
            Ah = round_complex(u, "fp16") * s[:, None, None, None]
            Y = coarse_op_apply(Ah, xh, L, disp) + 2.0 ** -11 * coarse_op_apply(Ah, xl, L, disp)
        else:
            ah, al = split16_complex(round_complex(u, "fp32"))
            ah, al = ah * s[:, None, None, None], al * s[:, None, None, None]
            Y = (coarse_op_apply(ah, xh, L, disp) + 2.0 ** -11 * coarse_op_apply(ah, xl, L, disp)
                 + 2.0 ** -11 * coarse_op_apply(al, xh, L, disp))
        return Y + site_diagonal(A)[:, None, None] * X32
    s = site_scales(A)
    Ahat = round_complex(remainder(A) / s[:, None, None, None], kind) * s[:, None, None, None]
    X32 = round_complex(X, "fp32")
    return coarse_op_apply(Ahat, quantise_vec(X, kind), L, disp) + \
        site_diagonal(A)[:, None, None] * X32
