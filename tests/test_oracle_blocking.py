"""Pins of the oracle's block project / promote: the block-diagonal dense
matrix assembled with scipy (a different route), the adjoint identity,
project after promote is the identity for a block-orthonormal basis, and an
identity basis maps fine blocks to coarse sites unchanged."""
import numpy as np
import scipy.linalg

from oracle.blocking import block_project, block_promote


def basis_and_vectors(rng, nblk=5, vb=12, nbasis=4, R=3):
    B = rng.standard_normal((nblk, vb, nbasis)) + 1j * rng.standard_normal((nblk, vb, nbasis))
    F = rng.standard_normal((nblk, vb, R)) + 1j * rng.standard_normal((nblk, vb, R))
    C = rng.standard_normal((nblk, nbasis, R)) + 1j * rng.standard_normal((nblk, nbasis, R))
    return B, F, C


def test_matches_block_diagonal_matrix(rng):
    B, F, C = basis_and_vectors(rng)
    P = scipy.linalg.block_diag(*B)          # (nblk vb) x (nblk nbasis)
    R = F.shape[-1]
    assert np.allclose(block_promote(B, C).reshape(-1, R), P @ C.reshape(-1, R), atol=1e-13)
    assert np.allclose(block_project(B, F).reshape(-1, R), np.conj(P).T @ F.reshape(-1, R),
                       atol=1e-13)


def test_adjoint_identity(rng):
    B, F, C = basis_and_vectors(rng, nblk=3, vb=16, nbasis=6, R=2)
    lhs = np.vdot(F, block_promote(B, C))
    rhs = np.vdot(block_project(B, F), C)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_orthonormal_basis_round_trip(rng):
    B, F, C = basis_and_vectors(rng, nblk=4, vb=20, nbasis=8, R=5)
    Q = np.stack([np.linalg.qr(b)[0] for b in B])
    assert np.allclose(block_project(Q, block_promote(Q, C)), C, atol=1e-12)
    # promote after project is the orthogonal projector onto the basis span
    Pf = block_promote(Q, block_project(Q, F))
    assert np.allclose(block_promote(Q, block_project(Q, Pf)), Pf, atol=1e-12)


def test_identity_basis(rng):
    nblk, n, R = 3, 6, 4
    eye = np.broadcast_to(np.eye(n, dtype=np.complex128), (nblk, n, n))
    F = rng.standard_normal((nblk, n, R)) + 1j * rng.standard_normal((nblk, n, R))
    assert np.array_equal(block_project(eye, F), F)
    assert np.array_equal(block_promote(eye, F), F)
