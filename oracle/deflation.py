"""Deflated Chebyshev coarse solve Q^{Cheby+defl} (Sec. 2.3, "two step
deflated/Chebyshev coarse solve").

Test infrastructure only (see the package docstring).

With the n_ev lowest eigenpairs (lambda_i, |i>) of the Hermitian coarse
operator H, a source b is split into its parts parallel and perpendicular to
the deflation space, b = b_par + b_perp, b_par = sum_i |i><i| b.  The
parallel part is inverted exactly, sum_i |i><i| b / lambda_i, and the
perpendicular part goes through the Chebyshev approximation P of 1/x on
[lo, hi]:
    Q b = sum_i |i> <i|b> / lambda_i + P(H) (b - sum_i |i><i|b>).
In H's eigenbasis Q is diagonal with entries 1/lambda_i on the deflated
modes and P(lambda_j) on the others.

Layouts: U is [V][nb][n_ev] (column i = eigenvector i, the same layout as a
block of n_ev right-hand sides), lam has n_ev entries, B is [V][nb][R].
"""
import numpy as np

from .ops import as_matrix
from .solvers import cheby_apply


def deflate_split(U, lam, B):
    """(sum_i |i><i|b>/lambda_i, b - sum_i |i><i|b>) for every column b of B:
    the two GEMMs of the deflation step, G = U^dagger B (n_ev x R) then
    U Lambda^-1 G and B - U G."""
    Bm = as_matrix(B)
    Um = U.reshape(Bm.shape[0], -1) if U.size else np.zeros((Bm.shape[0], 0), np.complex128)
    G = np.conj(Um).T @ Bm
    lam = np.asarray(lam, dtype=np.float64)
    par = Um @ (G / lam[:, None])
    perp = Bm - Um @ G
    return par.reshape(B.shape), perp.reshape(B.shape)


def defl_cheby_apply(apply_H, U, lam, B, lo, hi, order):
    """Q^{Cheby+defl} B: the exact inverse on the deflation space plus the
    degree-`order` Chebyshev approximation of 1/x on [lo, hi] applied to the
    perpendicular part."""
    par, perp = deflate_split(U, lam, B)
    return par + cheby_apply(apply_H, perp, lo, hi, order)
