"""Pins of the oracle's Cholesky, BlockCGrQ, Preconditioned BlockCGrQ,
Chebyshev polynomial, CG and spectral estimates.

Independent references: LAPACK (numpy) Cholesky and dense solves, plain CG
with one RHS, finite termination of block CG in ceil(N/nrhs) steps, the
recurrence invariants of Fig. 2, the convergence bound of Eq. (bound), and
the closed form 1 - x p(x) = T_{m+1}(t(x)) / T_{m+1}(t(0)) of the
Chebyshev interpolant of 1/x.
"""
import numpy as np
import pytest

from oracle.chol import Breakdown, chol_upper, hpd_inverse, upper_inverse
from oracle.ops import coarse_op_apply, column_norms
from oracle.solvers import (block_cg_rq, cg, cheby_apply, cheby_coeffs, cheby_eval_scalar,
                            lanczos_extremes, power_method, prec_block_cg_rq)
from synth import coarse_op, stencil, vectors
from tests.test_oracle_ops import dense_matrix


def problem(L, nb, npts, kappa, seed):
    """Generated operator with its shift set from the exact dense spectrum."""
    disp, _ = stencil(npts)
    A0 = coarse_op(L, nb, npts, seed, 0.0)
    ev = np.linalg.eigvalsh(dense_matrix(A0, L, disp))
    c = (ev[-1] - kappa * ev[0]) / (kappa - 1)
    A = coarse_op(L, nb, npts, seed, c)
    H = dense_matrix(A, L, disp)
    return A, H, disp


def test_cholesky_against_lapack(rng):
    for n in (1, 4, 17, 32):
        W = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
        G = W @ np.conj(W.T) + 0.1 * np.eye(n)
        S = chol_upper(G)
        Lc = np.linalg.cholesky(G)
        assert np.allclose(S, np.conj(Lc.T), atol=1e-10)
        assert np.allclose(np.triu(S), S)
        assert np.all(np.real(np.diag(S)) > 0) and np.allclose(np.imag(np.diag(S)), 0)
        assert np.allclose(upper_inverse(S) @ S, np.eye(n), atol=1e-9)
        assert np.allclose(hpd_inverse(G), np.linalg.inv(G), atol=1e-8)


def test_cholesky_breakdown_on_rank_deficiency(rng):
    W = rng.standard_normal((6, 3)) + 1j * rng.standard_normal((6, 3))
    W = np.concatenate([W, W[:, :1]], axis=1)        # duplicated column
    with pytest.raises(Breakdown):
        chol_upper(np.conj(W.T) @ W)


def test_block_cg_matches_dense_solve():
    L, nb, R = (2, 3, 2, 2), 3, 4
    A, H, disp = problem(L, nb, 81, 1e3, 101)
    B = vectors(L, nb, R, 101)
    X, info = block_cg_rq(lambda V: coarse_op_apply(A, V, L, disp), B, tol=1e-12, maxiter=500)
    ref = np.linalg.solve(H, B.reshape(-1, R)).reshape(B.shape)
    assert info["converged"] and np.all(info["resid"] <= 1e-11)
    assert np.linalg.norm(X - ref) <= 1e3 * 1e-11 * np.linalg.norm(ref)


def test_single_rhs_block_cg_equals_cg():
    L, nb = (2, 2, 3, 2), 2
    A, H, disp = problem(L, nb, 9, 1e2, 202)
    b = vectors(L, nb, 1, 202)
    op = lambda V: coarse_op_apply(A, V, L, disp)  # noqa: E731
    hb = []
    block_cg_rq(op, b, tol=1e-14, maxiter=30, history=hb)
    hc = []
    cg(lambda v: (H @ v.reshape(-1)), b.reshape(-1), tol=1e-14, maxiter=30, history=hc)
    n = min(len(hb), len(hc), 20)
    assert n >= 10
    for k in range(n):
        xb = hb[k]["X"].reshape(-1)
        xc = hc[k]["x"]
        assert np.linalg.norm(xb - xc) <= 1e-10 * np.linalg.norm(xc)


def test_finite_termination():
    """N = 32 unknowns, 4 RHS, kappa = 1e6: exact arithmetic terminates after
    N / nrhs = 8 block steps; allow two extra for rounding."""
    L, nb, R = (2, 2, 2, 2), 2, 4
    A, H, disp = problem(L, nb, 81, 1e6, 303)
    B = vectors(L, nb, R, 303)
    X, info = block_cg_rq(lambda V: coarse_op_apply(A, V, L, disp), B, tol=1e-8, maxiter=50)
    assert info["converged"] and info["iters"] <= 32 // R + 2


def test_block_cg_recurrence_invariants():
    L, nb, R = (2, 3, 2, 2), 3, 3
    A, H, disp = problem(L, nb, 9, 1e3, 404)
    B = vectors(L, nb, R, 404)
    hist = []
    block_cg_rq(lambda V: coarse_op_apply(A, V, L, disp), B, tol=1e-12, maxiter=12, history=hist)
    Bm = B.reshape(-1, R)
    for h in hist[:8]:
        res = Bm - H @ h["X"]
        assert np.allclose(res, h["Q"] @ h["C"], atol=1e-9 * np.linalg.norm(Bm))
        assert np.allclose(np.conj(h["Q"].T) @ h["Q"], np.eye(R), atol=1e-8)
    # block H-conjugacy of successive search directions D_j^dagger H D_k = 0
    Ds = [h["D"] for h in hist[:5]]
    for j in range(len(Ds) - 1):
        cross = np.conj(Ds[j].T) @ H @ Ds[j + 1]
        assert np.linalg.norm(cross) <= 1e-7 * np.linalg.norm(Ds[j]) * np.linalg.norm(H @ Ds[j + 1])


def test_convergence_bound_free_laplacian():
    """Eq. (bound): the H-norm error of CG (and, column by column, of block
    CG, whose block Krylov space contains each single one) decays at least
    like 2 sigma^k with sigma = (sqrt(kappa) - 1)/(sqrt(kappa) + 1)."""
    L = (6, 4, 4, 4)
    m2 = 0.05
    disp, _ = stencil(9)
    V = int(np.prod(L))
    A = np.zeros((V, 9, 1, 1), dtype=np.complex128)
    A[:, 0] = 8.0 + m2
    A[:, 1:] = -1.0
    lam_max = m2 + sum(2 - 2 * np.cos(2 * np.pi * (l // 2) / l) for l in L)
    kappa = lam_max / m2
    sigma = (np.sqrt(kappa) - 1) / (np.sqrt(kappa) + 1)
    H = dense_matrix(A, L, disp)
    B = vectors(L, 1, 3, 505)
    xs = np.linalg.solve(H, B.reshape(-1, 3))
    enorm = lambda e: np.sqrt(np.real(np.sum(np.conj(e) * (H @ e), axis=0)))  # noqa: E731
    e0 = enorm(xs)
    hist = []
    block_cg_rq(lambda Vv: coarse_op_apply(A, Vv, L, disp), B, tol=1e-12, maxiter=60, history=hist)
    for k, h in enumerate(hist[:40], start=1):
        ek = enorm(xs - h["X"])
        assert np.all(ek <= 2 * sigma ** k * e0 * (1 + 1e-8) + 1e-12)
    hc = []
    cg(lambda v: H @ v, B.reshape(-1, 3)[:, 0], tol=1e-12, maxiter=60, history=hc)
    for k, h in enumerate(hc[:40], start=1):
        ek = enorm((xs[:, 0] - h["x"])[:, None])[0]
        assert ek <= 2 * sigma ** k * e0[0] * (1 + 1e-8) + 1e-12


@pytest.mark.parametrize("lo,hi,m", [(0.5, 40.0, 8), (0.02, 40.0, 120), (2.0, 92.0, 8), (1.0, 3.0, 0)])
def test_chebyshev_residual_closed_form(lo, hi, m):
    lam = np.concatenate([np.linspace(lo, hi, 41), [0.3 * lo, 0.9 * lo, 1e-3 * lo]])
    p = cheby_eval_scalar(lam, lo, hi, m)
    t = lambda x: (2 * x - (hi + lo)) / (hi - lo)  # noqa: E731
    from oracle.solvers import _cheb_T
    ref = _cheb_T(m + 1, t(lam)) / _cheb_T(m + 1, t(np.array([0.0])))[0]
    assert np.allclose(1 - lam * p, ref, atol=1e-9)
    # worst case on [lo, hi] is 1/|T_{m+1}(t(0))|; p > 0 below hi
    bound = 1.0 / abs(_cheb_T(m + 1, t(np.array([0.0])))[0])
    assert np.all(np.abs(1 - lam[:41] * p[:41]) <= bound * (1 + 1e-9))
    assert np.all(p > 0)


def test_chebyshev_apply_on_diagonal_operator():
    lam = np.linspace(0.7, 30.0, 23)
    V = (np.arange(23) + 1.0)[:, None] * np.ones((1, 2)) + 0j
    out = cheby_apply(lambda X: lam[:, None] * X, V, 0.5, 32.0, 17)
    ref = cheby_eval_scalar(lam, 0.5, 32.0, 17)[:, None] * V
    assert np.allclose(out, ref, rtol=1e-11, atol=0)
    assert len(cheby_coeffs(0.5, 32.0, 17)) == 18


def test_prec_block_cg_special_cases():
    L, nb, R = (2, 2, 3, 2), 2, 3
    A, H, disp = problem(L, nb, 81, 1e3, 606)
    B = vectors(L, nb, R, 606)
    op = lambda V: coarse_op_apply(A, V, L, disp)  # noqa: E731
    # M = identity reproduces BlockCGrQ iterate by iterate
    h1, h2 = [], []
    block_cg_rq(op, B, tol=1e-13, maxiter=10, history=h1)
    prec_block_cg_rq(op, lambda V: V, B, tol=1e-13, maxiter=10, history=h2)
    for a, b in zip(h1[:8], h2[:8]):
        assert np.linalg.norm(a["X"] - b["X"]) <= 1e-9 * np.linalg.norm(a["X"])
    # M^-1 = H^-1 (exact): one step
    Hinv = np.linalg.inv(H)
    X, info = prec_block_cg_rq(op, lambda V: (Hinv @ V.reshape(-1, V.shape[-1])).reshape(V.shape),
                               B, tol=1e-10, maxiter=5)
    assert info["converged"] and info["iters"] == 1


def test_prec_block_cg_chebyshev_invariants():
    L, nb, R = (2, 3, 2, 2), 3, 4
    A, H, disp = problem(L, nb, 81, 1e3, 707)
    B = vectors(L, nb, R, 707)
    op = lambda V: coarse_op_apply(A, V, L, disp)  # noqa: E731
    ev = np.linalg.eigvalsh(H)
    lo, hi = 10 * ev[0], 1.1 * ev[-1]
    Minv = lambda V: cheby_apply(op, V, lo, hi, 6)  # noqa: E731
    hist = []
    X, info = prec_block_cg_rq(op, Minv, B, tol=1e-10, maxiter=200, history=hist)
    assert info["converged"]
    Bm = B.reshape(-1, R)
    for h in hist[:6]:
        res = Bm - H @ h["X"]
        assert np.allclose(res, h["q"] @ h["C"], atol=1e-9 * np.linalg.norm(Bm))
        assert np.allclose(np.conj(h["Q"].T) @ h["q"], np.eye(R), atol=1e-8)
    ref = np.linalg.solve(H, Bm)
    assert np.linalg.norm(X.reshape(-1, R) - ref) <= 1e3 * 1e-9 * np.linalg.norm(ref)


def test_chebyshev_preconditioning_cuts_outer_iterations():
    L, nb, R = (4, 4, 3, 3), 4, 2
    A, H, disp = problem(L, nb, 9, 1e3, 717)
    B = vectors(L, nb, R, 717)
    op = lambda V: coarse_op_apply(A, V, L, disp)  # noqa: E731
    ev = np.linalg.eigvalsh(H)
    Xp, ip = prec_block_cg_rq(op, lambda V: cheby_apply(op, V, ev[0], 1.1 * ev[-1], 16), B,
                              tol=1e-9, maxiter=500)
    Xb, ib = block_cg_rq(op, B, tol=1e-9, maxiter=500)
    assert ip["converged"] and ib["converged"]
    assert 3 * ip["iters"] < ib["iters"]
    ref = np.linalg.solve(H, B.reshape(-1, R))
    for X in (Xp, Xb):
        assert np.linalg.norm(X.reshape(-1, R) - ref) <= 1e3 * 1e-8 * np.linalg.norm(ref)


def test_rank_deficient_block():
    """Duplicated and linearly dependent right-hand sides narrow the block."""
    L, nb = (2, 3, 2, 2), 3
    A, H, disp = problem(L, nb, 81, 1e3, 727)
    B = vectors(L, nb, 4, 727)
    B[:, :, 2] = B[:, :, 0]
    B[:, :, 3] = 0.5 * B[:, :, 1] - 2j * B[:, :, 0]
    op = lambda V: coarse_op_apply(A, V, L, disp)  # noqa: E731
    for solver in (lambda: block_cg_rq(op, B, tol=1e-10, maxiter=200),
                   lambda: prec_block_cg_rq(op, lambda V: cheby_apply(op, V, 0.1, 40.0, 4), B,
                                            tol=1e-10, maxiter=200)):
        X, info = solver()
        assert info["converged"] and np.all(info["resid"] <= 1e-9)


def test_zero_column():
    L, nb = (2, 2, 2, 2), 2
    A, H, disp = problem(L, nb, 9, 1e2, 808)
    B = vectors(L, nb, 3, 808)
    B[:, :, 1] = 0.0
    X, info = block_cg_rq(lambda V: coarse_op_apply(A, V, L, disp), B, tol=1e-10)
    assert np.all(X[:, :, 1] == 0) and info["converged"]


def test_spectral_estimates():
    L, nb = (3, 2, 2, 2), 3
    A, H, disp = problem(L, nb, 81, 1e3, 909)
    ev = np.linalg.eigvalsh(H)
    op = lambda v: coarse_op_apply(A, v.reshape(-1, nb, 1), L, disp).reshape(-1)  # noqa: E731
    v0 = vectors(L, nb, 1, 909, stream=6).reshape(-1)
    lmax = power_method(op, v0, iters=300)
    assert abs(lmax - ev[-1]) <= 2e-2 * ev[-1]
    tmin, tmax, bmin, bmax = lanczos_extremes(op, v0, 72)
    assert abs(tmin - ev[0]) <= 1e-8 * ev[-1] and abs(tmax - ev[-1]) <= 1e-8 * ev[-1]
    assert tmin >= ev[0] - 1e-10 and tmax <= ev[-1] + 1e-10
    assert column_norms(np.ones((4, 2))).shape == (2,)
