"""Pins of the oracle's coarsening: identity blocking returns the fine
operator, the Galerkin identity (coarse operator = P^dagger M P through the
pinned block projector and operator), Hermiticity carried to the coarse
operator, and the momentum-phase method equal to the definition."""
import numpy as np
import pytest

from oracle.coarsen import coarsen_direct, coarsen_phase, galerkin_apply
from oracle.ops import coarse_op_apply
from synth import coarse_op, stencil, vectors


def fine_problem(Lf, nbf, seed, shift=6.0):
    disp, _ = stencil(81)
    A = coarse_op(Lf, nbf, 81, seed, shift)
    return disp, A, (lambda X: coarse_op_apply(A, X, Lf, disp))


def random_basis(rng, Vc, vb, nbasis):
    B = rng.standard_normal((Vc, vb, nbasis)) + 1j * rng.standard_normal((Vc, vb, nbasis))
    return np.stack([np.linalg.qr(b)[0] for b in B])


def test_identity_blocking_returns_the_fine_operator():
    Lf, nbf = (3, 3, 3, 4), 2
    disp, A, M = fine_problem(Lf, nbf, 71)
    V = int(np.prod(Lf))
    basis = np.broadcast_to(np.eye(nbf, dtype=np.complex128), (V, nbf, nbf)).copy()
    Ac = coarsen_direct(M, Lf, nbf, (1, 1, 1, 1), basis, disp)
    assert np.allclose(Ac, A, atol=1e-13)
    Ap = coarsen_phase(M, Lf, nbf, (1, 1, 1, 1), basis, disp)
    assert np.allclose(Ap, A, atol=1e-11)


@pytest.mark.parametrize("block", [(2, 1, 1, 2), (1, 2, 2, 1)])
def test_galerkin_hermiticity_and_phase_method(rng, block):
    Lc, nbf, nbasis = (3, 3, 3, 3), 2, 3
    Lf = tuple(l * b for l, b in zip(Lc, block))
    disp, A, M = fine_problem(Lf, nbf, 72 + block[0])
    Vc, vb = int(np.prod(Lc)), int(np.prod(block)) * nbf
    basis = random_basis(rng, Vc, vb, nbasis)
    Ac = coarsen_direct(M, Lf, nbf, block, basis, disp)
    C = vectors(Lc, nbasis, 2, 73)
    assert np.allclose(coarse_op_apply(Ac, C, Lc, disp), galerkin_apply(M, Lf, block, basis, C),
                       atol=1e-12)
    # Hermitian fine operator -> A_{-p}(b + delta_p) = A_p(b)^dagger
    _, pair = stencil(81)
    from oracle.coarsen import coarse_neighbours
    nbr = coarse_neighbours(Lc, disp)
    for p in range(81):
        assert np.allclose(Ac[nbr[p], pair[p]], np.conj(np.swapaxes(Ac[:, p], -1, -2)), atol=1e-12)
    Ap = coarsen_phase(M, Lf, nbf, block, basis, disp)
    assert np.allclose(Ap, Ac, atol=1e-11)
