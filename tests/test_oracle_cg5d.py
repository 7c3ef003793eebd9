"""Pins of the oracle's five-dimensional CG (one Krylov space for all
right-hand sides): the dense solution, the residual recurrence, finite
termination, and duplicated columns reproducing single-vector CG."""
import numpy as np

from oracle.ops import coarse_op_apply
from oracle.solvers import cg, cg5d
from synth import coarse_op, stencil, vectors

from test_oracle_ops import dense_matrix


def problem(L=(2, 2, 2, 3), nb=3, npts=81, shift=17.5, seed=55):
    disp, _ = stencil(npts)
    A = coarse_op(L, nb, npts, seed, shift)
    return A, L, disp, lambda X: coarse_op_apply(A, X, L, disp)


def test_dense_solution_and_recurrence():
    A, L, disp, H = problem()
    H0 = dense_matrix(A, L, disp)
    assert np.linalg.eigvalsh(H0)[0] > 0
    B = vectors(L, 3, 4, 56)
    hist = []
    X, info = cg5d(H, B, tol=1e-11, maxiter=500, history=hist)
    N = H0.shape[0]
    ref = np.linalg.solve(H0, B.reshape(N, -1)).reshape(B.shape)
    assert np.max(info["resid"]) <= 1e-10
    assert np.allclose(X, ref, atol=1e-9 * np.abs(ref).max())
    for h in hist[::5]:      # the updated residual is the true one
        true = (B - H(h["X"].reshape(B.shape))).reshape(N, -1)
        assert np.allclose(h["r"], true, atol=1e-9 * np.abs(B).max())


def test_finite_termination():
    # N = 16 unknowns: the enlarged operator has at most 16 distinct eigenvalues
    A, L, disp, H = problem(L=(2, 2, 1, 2), nb=2, shift=20.0, seed=57)
    B = vectors(L, 2, 3, 58)
    X, info = cg5d(H, B, tol=1e-10, maxiter=200)
    assert info["iters"] <= 16 + 2 and np.max(info["resid"]) <= 1e-9


def test_duplicated_columns_reproduce_single_cg():
    A, L, disp, H = problem(seed=59)
    b = vectors(L, 3, 1, 60)
    B = np.concatenate([b, b], axis=2)
    h5, h1 = [], []
    X, info = cg5d(H, B, tol=1e-12, maxiter=40, history=h5)
    x, i1 = cg(lambda v: H(v.reshape(b.shape)).reshape(-1), b, tol=1e-12, maxiter=40, history=h1)
    n = min(len(h5), len(h1))
    assert n >= 10
    for k in range(n):
        assert np.allclose(h5[k]["X"][:, 0], h1[k]["x"], atol=1e-12 * np.abs(x).max())
        assert np.allclose(h5[k]["X"][:, 1], h1[k]["x"], atol=1e-12 * np.abs(x).max())
