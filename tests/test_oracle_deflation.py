"""Pins of the oracle's deflated Chebyshev coarse solve against the spectral
decomposition of small coarse operators (dense eigh, a different route):
eigenvectors inside the deflation space are inverted exactly, those outside
are scaled by the Chebyshev polynomial evaluated as a scalar, all
eigenvectors deflated gives H^-1, none gives the plain polynomial, and Q is
Hermitian."""
import numpy as np
import pytest

from oracle.deflation import defl_cheby_apply, deflate_split
from oracle.ops import coarse_op_apply
from oracle.solvers import cheby_apply, cheby_eval_scalar
from synth import coarse_op, stencil, vectors

from test_oracle_ops import dense_matrix


@pytest.fixture(scope="module")
def small():
    L, nb, npts = (2, 2, 3, 2), 3, 81
    disp, _ = stencil(npts)
    A = coarse_op(L, nb, npts, 4711, 17.5)   # lambda_min ~ 0.3
    H = dense_matrix(A, L, disp)
    lam, W = np.linalg.eigh(H)
    assert lam[0] > 0
    V = int(np.prod(L))
    apply_H = lambda X: coarse_op_apply(A, X, L, disp)
    return dict(L=L, nb=nb, V=V, A=A, H=H, lam=lam, W=W, apply_H=apply_H)


def as_block(W, V, nb):
    return W.reshape(V, nb, -1)


def test_eigenvectors_inverted_or_polynomial(small):
    s = small
    n_ev, lo, hi, order = 10, s["lam"][10] / 2, 1.05 * s["lam"][-1], 24
    U = as_block(s["W"][:, :n_ev], s["V"], s["nb"])
    for j in (0, 3, 9, 10, 25, len(s["lam"]) - 1):
        B = as_block(s["W"][:, j:j + 1], s["V"], s["nb"])
        Q = defl_cheby_apply(s["apply_H"], U, s["lam"][:n_ev], B, lo, hi, order)
        want = 1.0 / s["lam"][j] if j < n_ev else cheby_eval_scalar(s["lam"][j], lo, hi, order)
        assert np.allclose(Q, want * B, atol=1e-11 * abs(want))


def test_all_deflated_is_the_inverse(small):
    s = small
    N = len(s["lam"])
    U = as_block(s["W"], s["V"], s["nb"])
    B = vectors(s["L"], s["nb"], 4, 17)
    Q = defl_cheby_apply(s["apply_H"], U, s["lam"], B, 1.0, 2.0, 5)
    ref = np.linalg.solve(s["H"], B.reshape(N, -1)).reshape(B.shape)
    assert np.allclose(Q, ref, atol=1e-10 * np.abs(ref).max())


def test_nothing_deflated_is_the_polynomial(small):
    s = small
    B = vectors(s["L"], s["nb"], 3, 18)
    U = np.zeros((s["V"], s["nb"], 0), dtype=np.complex128)
    lo, hi, order = 0.5, 1.05 * s["lam"][-1], 16
    Q = defl_cheby_apply(s["apply_H"], U, np.zeros(0), B, lo, hi, order)
    assert np.allclose(Q, cheby_apply(s["apply_H"], B, lo, hi, order), atol=1e-13)
    # and the polynomial through the spectral decomposition
    N = len(s["lam"])
    p = cheby_eval_scalar(s["lam"], lo, hi, order)
    ref = (s["W"] @ (p[:, None] * (np.conj(s["W"]).T @ B.reshape(N, -1)))).reshape(B.shape)
    assert np.allclose(Q, ref, atol=1e-11 * np.abs(ref).max())


def test_split_and_hermiticity(small, rng):
    s = small
    n_ev = 7
    U = as_block(s["W"][:, :n_ev], s["V"], s["nb"])
    B = vectors(s["L"], s["nb"], 2, 19)
    par, perp = deflate_split(U, s["lam"][:n_ev], B)
    # perp is orthogonal to the deflation space; par solves H x = b_par
    Um = U.reshape(-1, n_ev)
    assert np.abs(np.conj(Um).T @ perp.reshape(-1, 2)).max() < 1e-12
    Bpar = B - perp
    assert np.allclose(s["apply_H"](par), Bpar, atol=1e-11)
    u = vectors(s["L"], s["nb"], 1, 20)
    v = vectors(s["L"], s["nb"], 1, 21)
    lo, hi, order = s["lam"][n_ev] / 2, 1.05 * s["lam"][-1], 12
    Qv = defl_cheby_apply(s["apply_H"], U, s["lam"][:n_ev], v, lo, hi, order)
    Qu = defl_cheby_apply(s["apply_H"], U, s["lam"][:n_ev], u, lo, hi, order)
    assert abs(np.vdot(u, Qv) - np.vdot(Qu, v)) < 1e-11 * abs(np.vdot(u, Qv))
