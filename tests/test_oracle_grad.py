"""Pins of the oracle adjoints: central finite differences of a real loss
along random directions (any direction for the operator; Hermitian-preserving
directions for the solve, which needs a Hermitian operator)."""
import numpy as np

from oracle.grad import op_vjp, solve_vjp
from oracle.ops import coarse_op_apply
from synth import coarse_op, stencil, vectors
from tests.test_oracle_ops import dense_matrix


def hermitian_direction(L, nb, npts, rng):
    """Random perturbation field with D_{-p}(x + delta_p) = D_p(x)^dagger."""
    from synth.coarse import shifted_sites
    disp, pair = stencil(npts)
    V = int(np.prod(L))
    D = rng.standard_normal((V, npts, nb, nb)) + 1j * rng.standard_normal((V, npts, nb, nb))
    D[:, 0] = 0.5 * (D[:, 0] + np.conj(np.swapaxes(D[:, 0], -1, -2)))
    for p in range(npts):
        if p != 0 and pair[p] > p:
            continue
        if p == 0:
            continue
        q = pair[p]
        y = shifted_sites(L, np.arange(V), disp[q])
        D[y, p] = np.conj(np.swapaxes(D[:, q], -1, -2))
    return D


def test_operator_vjp_finite_differences(rng):
    L, nb, npts, R = (3, 2, 2, 2), 3, 81, 2
    disp, _ = stencil(npts)
    A = coarse_op(L, nb, npts, 5, 4.0)
    X = vectors(L, nb, R, 5)
    w = vectors(L, nb, R, 6)
    loss = lambda A_, X_: np.real(np.sum(w * coarse_op_apply(A_, X_, L, disp)))  # noqa: E731
    GY = np.conj(w)
    GA, GX = op_vjp(A, X, GY, L, disp)
    h = 1e-6
    for _ in range(4):
        dA = rng.standard_normal(A.shape) + 1j * rng.standard_normal(A.shape)
        dX = rng.standard_normal(X.shape) + 1j * rng.standard_normal(X.shape)
        fd = (loss(A + h * dA, X + h * dX) - loss(A - h * dA, X - h * dX)) / (2 * h)
        an = np.real(np.sum(np.conj(GA) * dA) + np.sum(np.conj(GX) * dX))
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an))


def test_solve_vjp_finite_differences(rng):
    L, nb, npts, R = (2, 3, 2, 2), 3, 9, 2
    disp, _ = stencil(npts)
    A = coarse_op(L, nb, npts, 7, 7.0)
    B = vectors(L, nb, R, 7)
    w = vectors(L, nb, R, 8)
    N = int(np.prod(L)) * nb

    def solve_with(A_, B_):
        H = dense_matrix(A_, L, disp)
        return np.linalg.solve(H, B_.reshape(N, R)).reshape(B_.shape)

    loss = lambda A_, B_: np.real(np.sum(w * solve_with(A_, B_)))  # noqa: E731
    X = solve_with(A, B)
    GA, GB = solve_vjp(lambda G: solve_with(A, G), X, np.conj(w), L, disp)
    h = 1e-6
    for _ in range(4):
        dA = hermitian_direction(L, nb, npts, rng)
        dB = rng.standard_normal(B.shape) + 1j * rng.standard_normal(B.shape)
        fd = (loss(A + h * dA, B + h * dB) - loss(A - h * dA, B - h * dB)) / (2 * h)
        an = np.real(np.sum(np.conj(GA) * dA) + np.sum(np.conj(GB) * dB))
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an))
    # the perturbation generator keeps the operator Hermitian
    H = dense_matrix(A + 0.1 * hermitian_direction(L, nb, npts, rng), L, disp)
    assert np.allclose(H, np.conj(H.T))
