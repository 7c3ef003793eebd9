"""Pins of the oracle's two-level ADEF2 preconditioner and flexible ADEF2 CG
(Fig. 1), on small dense problems:

* Galerkin algebra: Q H Q = Q, and the start x_0 = Q b + P_R x has a
  residual orthogonal to the coarse space for any x;
* a complete coarse space (the basis spans every degree of freedom) makes
  Q = H^-1, so the start already solves the system; an exact smoother makes
  M^-1 = H^-1, so one iteration solves it;
* M^-1 = I, Q = 0 reduces flexible ADEF2 to plain CG, iterate by iterate
  (with and without the flexible orthogonalisation, whose coefficients
  vanish for a fixed preconditioner);
* with a variable preconditioner (a few CG steps) the orthogonalisation
  keeps each search direction H-conjugate to the previous one;
* the fixed-iteration CG smoother reaches the exact solution once the
  iteration count passes the dimension (finite termination), and the
  deflated guess with every eigenvector is the exact inverse.
"""
import numpy as np
import pytest

from oracle.ops import coarse_op_apply
from oracle.solvers import cg
from oracle.twolevel import (adef2_apply, cg_fixed, cg_to_tol, deflated_guess, flex_adef2,
                             flex_adef2_columns)
from synth import coarse_op, stencil, vectors
from tests.test_oracle_ops import dense_matrix


def setup(nbasis, seed=3):
    L, nb, npts = (2, 2, 2, 2), 3, 9
    disp, _ = stencil(npts)
    A = coarse_op(L, nb, npts, seed, 9.0)
    H = dense_matrix(A, L, disp)
    N = H.shape[0]
    rng = np.random.default_rng(seed)
    # blocks of two sites (6 degrees of freedom), an orthonormal basis of
    # nbasis vectors per block: P is N x (8 nbasis)
    nblk, vb = N // 6, 6
    P = np.zeros((N, nblk * nbasis), dtype=np.complex128)
    for k in range(nblk):
        G = rng.standard_normal((vb, nbasis)) + 1j * rng.standard_normal((vb, nbasis))
        q, _ = np.linalg.qr(G)
        P[k * vb:(k + 1) * vb, k * nbasis:(k + 1) * nbasis] = q
    h = np.conj(P.T) @ H @ P
    Q = P @ np.linalg.solve(h, np.conj(P.T))
    return H, P, Q, rng, (A, L, disp)


def test_galerkin_algebra():
    H, P, Q, rng, _ = setup(2)
    assert np.linalg.norm(Q @ H @ Q - Q) <= 1e-12 * np.linalg.norm(Q)
    b = rng.standard_normal(H.shape[0]) + 1j * rng.standard_normal(H.shape[0])
    x = rng.standard_normal(H.shape[0]) + 1j * rng.standard_normal(H.shape[0])
    x0 = Q @ b + x - Q @ (H @ x)
    assert np.linalg.norm(np.conj(P.T) @ (b - H @ x0)) <= 1e-12 * np.linalg.norm(b)
    # P_R Q = 0: the smoother's correction never undoes the coarse one
    PR = np.eye(H.shape[0]) - Q @ H
    assert np.linalg.norm(PR @ Q) <= 1e-12 * np.linalg.norm(Q)


def test_complete_space_and_exact_smoother():
    H, P, Q, rng, _ = setup(6)                    # six basis vectors per 6-dof block
    N = H.shape[0]
    assert np.linalg.norm(Q - np.linalg.inv(H)) <= 1e-10 * np.linalg.norm(Q)
    b = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    x, info = flex_adef2(lambda v: H @ v, lambda r: r, lambda v: Q @ v, b, tol=1e-10)
    assert info["iters"] == 0 and info["resid"] <= 1e-10
    # any guess: x_0 = Q b + P_R x = H^-1 b as well
    xg = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    x, info = flex_adef2(lambda v: H @ v, lambda r: r, lambda v: Q @ v, b, x=xg, tol=1e-10)
    assert info["iters"] == 0 and info["resid"] <= 1e-10
    # a partial coarse space with an exact smoother: M^-1 = H^-1, one step
    H, P, Q, rng, _ = setup(2)
    Hinv = np.linalg.inv(H)
    M = lambda r: adef2_apply(lambda v: H @ v, lambda v: Hinv @ v, lambda v: Q @ v, r)  # noqa
    r = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    assert np.linalg.norm(M(r) - Hinv @ r) <= 1e-10 * np.linalg.norm(Hinv @ r)
    x, info = flex_adef2(lambda v: H @ v, M, lambda v: Q @ v, b, tol=1e-10)
    assert info["iters"] == 1 and info["resid"] <= 1e-10


@pytest.mark.parametrize("mmax", [0, 2])
def test_identity_preconditioner_is_plain_cg(mmax):
    H, P, Q, rng, _ = setup(2)
    N = H.shape[0]
    b = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    hist_f, hist_c = [], []
    xf, inf = flex_adef2(lambda v: H @ v, lambda r: r, lambda v: 0 * v, b, tol=1e-10,
                         maxiter=200, mmax=mmax, history=hist_f)
    xc, inc = cg(lambda v: H @ v, b, tol=1e-10, maxiter=200, history=hist_c)
    assert inf["iters"] == inc["iters"]
    for hf, hc in zip(hist_f[:30], hist_c[:30]):
        assert np.linalg.norm(hf["x"] - hc["x"]) <= 1e-9 * np.linalg.norm(hc["x"])


def test_variable_preconditioner_keeps_directions_conjugate():
    H, P, Q, rng, _ = setup(2)
    N = H.shape[0]
    b = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    # a variable preconditioner: three CG steps on H + 2 from x = 0
    Hs = H + 2.0 * np.eye(N)
    M = lambda r: cg_fixed(lambda v: Hs @ v, r, 3)  # noqa: E731
    hist = []
    x, info = flex_adef2(lambda v: H @ v, M, lambda v: 0 * v, b, tol=1e-10, maxiter=300,
                         mmax=1, history=hist)
    assert info["converged"]
    for prev, cur in zip(hist[:-1], hist[1:]):
        c = abs(np.vdot(cur["p"], prev["w"]))
        assert c <= 1e-9 * np.linalg.norm(cur["p"]) * np.linalg.norm(prev["w"])
        # w = H p holds after the orthogonalisation
        assert np.linalg.norm(cur["w"] - H @ cur["p"]) <= 1e-10 * np.linalg.norm(cur["w"])


def test_fixed_cg_finite_termination_and_deflated_guess():
    H, P, Q, rng, _ = setup(2)
    N = H.shape[0]
    b = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    x = cg_fixed(lambda v: H @ v, b, 3 * N)
    assert np.linalg.norm(H @ x - b) <= 1e-8 * np.linalg.norm(b)
    ev, U = np.linalg.eigh(H)
    assert np.linalg.norm(deflated_guess(U, ev, b) - np.linalg.solve(H, b)) <= \
        1e-10 * np.linalg.norm(np.linalg.solve(H, b))
    x2 = cg_to_tol(lambda v: H @ v, b, np.zeros(N), 1e-6, 500)
    assert np.linalg.norm(b - H @ x2) <= 1.1e-6 * np.linalg.norm(b)


def test_columns_and_lattice_operator():
    """flex_adef2_columns on a [V][nb][R] block with the lattice operator
    solves every column to tol against the oracle's operator."""
    H, P, Q, rng, (A, L, disp) = setup(2)
    R = 3
    B = vectors(L, 3, R, 77)
    shape = B.shape[:-1] + (1,)
    Hv = lambda v: coarse_op_apply(A, v.reshape(shape), L, disp).reshape(-1)  # noqa: E731
    X, infos = flex_adef2_columns(Hv, lambda r: r, lambda v: Q @ v, B, tol=1e-10, mmax=1)
    r = B - coarse_op_apply(A, X, L, disp)
    rel = np.linalg.norm(r.reshape(-1, R), axis=0) / np.linalg.norm(B.reshape(-1, R), axis=0)
    assert np.max(rel) <= 1e-9 and all(i["converged"] for i in infos)
