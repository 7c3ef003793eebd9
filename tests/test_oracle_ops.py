"""Pins of the oracle's coarse operator, adjoint, Gram and block update.

Each check compares the oracle with something other than itself: a densely
assembled matrix (built here by a different route), the momentum-space
closed form of a translation-invariant stencil, the free lattice Laplacian
spectrum, the V = 1 reduction to a single GEMM, the adjoint identity, and
plain numpy matrix products.
"""
import itertools

import numpy as np
import pytest

from oracle import native
from oracle.ops import block_axpy, block_inner, coarse_op_apply, coarse_op_apply_dag
from synth import coarse_op, stencil, vectors


def dense_matrix(A, L, disp):
    """Assemble H[x-block, y-block] += A_p(x) for y = x + delta_p, using
    numpy's multi-index routines instead of the oracle's neighbour table."""
    V, npts, nb, _ = A.shape
    H = np.zeros((V * nb, V * nb), dtype=np.complex128)
    dims = tuple(int(l) for l in L)
    for x in range(V):
        cx = np.array(np.unravel_index(x, dims, order="F"))
        for p in range(npts):
            cy = np.mod(cx + disp[p].astype(np.int64), dims)
            y = int(np.ravel_multi_index(tuple(cy), dims, order="F"))
            H[x * nb:(x + 1) * nb, y * nb:(y + 1) * nb] += A[x, p]
    return H


def random_general_op(L, nb, npts, rng):
    V = int(np.prod(L))
    return rng.standard_normal((V, npts, nb, nb)) + 1j * rng.standard_normal((V, npts, nb, nb))


@pytest.mark.parametrize("L,nb,npts,R", [((2, 3, 1, 2), 3, 9, 2), ((3, 3, 2, 2), 2, 81, 3),
                                         ((1, 1, 1, 1), 4, 81, 2), ((2, 2, 2, 2), 3, 81, 1)])
def test_op_matches_dense_assembly(L, nb, npts, R, rng):
    disp, _ = stencil(npts)
    A = random_general_op(L, nb, npts, rng)
    V = int(np.prod(L))
    X = rng.standard_normal((V, nb, R)) + 1j * rng.standard_normal((V, nb, R))
    H = dense_matrix(A, L, disp)
    ref = (H @ X.reshape(-1, R)).reshape(X.shape)
    assert np.allclose(coarse_op_apply(A, X, L, disp), ref, rtol=0, atol=1e-12)
    refd = (np.conj(H.T) @ X.reshape(-1, R)).reshape(X.shape)
    assert np.allclose(coarse_op_apply_dag(A, X, L, disp), refd, rtol=0, atol=1e-12)


def test_momentum_space_closed_form(rng):
    """Site-independent A_p: H e^{ik.x} v = e^{ik.x} (sum_p A_p e^{ik.delta_p}) v."""
    L = (4, 3, 5, 2)
    nb, npts = 3, 81
    disp, _ = stencil(npts)
    Ap = rng.standard_normal((npts, nb, nb)) + 1j * rng.standard_normal((npts, nb, nb))
    V = int(np.prod(L))
    A = np.broadcast_to(Ap, (V, npts, nb, nb)).copy()
    coords = np.array(list(itertools.product(*[range(l) for l in reversed(L)])))[:, ::-1]
    for n in [(0, 0, 0, 0), (1, 2, 3, 1), (3, 1, 4, 1)]:
        k = 2 * np.pi * np.array(n) / np.array(L)
        phase = np.exp(1j * coords @ k)                     # site order x0 fastest
        v = rng.standard_normal(nb) + 1j * rng.standard_normal(nb)
        X = (phase[:, None] * v[None, :])[:, :, None]
        Hk = np.einsum("pab,p->ab", Ap, np.exp(1j * disp.astype(np.float64) @ k))
        ref = (phase[:, None] * (Hk @ v)[None, :])[:, :, None]
        assert np.allclose(coarse_op_apply(A, X, L, disp), ref, atol=1e-11)


def test_free_laplacian_spectrum():
    """nb = 1, A_{+-mu} = -1, self 8 + m^2: eigenvalues m^2 + sum_mu (2 - 2 cos k_mu)."""
    L = (4, 4, 3, 5)
    m2 = 0.3
    disp, _ = stencil(9)
    V = int(np.prod(L))
    A = np.zeros((V, 9, 1, 1), dtype=np.complex128)
    A[:, 0] = 8.0 + m2
    A[:, 1:] = -1.0
    H = dense_matrix(A, L, disp)
    coords = np.array(list(itertools.product(*[range(l) for l in reversed(L)])))[:, ::-1]
    for n in [(0, 0, 0, 0), (1, 2, 1, 3), (2, 3, 2, 4)]:
        k = 2 * np.pi * np.array(n) / np.array(L)
        lam = m2 + np.sum(2 - 2 * np.cos(k))
        X = np.exp(1j * coords @ k)[:, None, None]
        assert np.allclose(coarse_op_apply(A, X, L, disp), lam * X, atol=1e-12)
    ev = np.sort(np.linalg.eigvalsh(H))
    ks = [np.sum(2 - 2 * np.cos(2 * np.pi * np.array(c) / np.array(L))) + m2
          for c in itertools.product(*[range(l) for l in L])]
    assert np.allclose(ev, np.sort(ks), atol=1e-11)


def test_single_site_is_one_gemm(rng):
    L = (1, 1, 1, 1)
    disp, _ = stencil(81)
    A = random_general_op(L, 5, 81, rng)
    X = rng.standard_normal((1, 5, 4)) + 1j * rng.standard_normal((1, 5, 4))
    ref = A[0].sum(axis=0) @ X[0]
    assert np.allclose(coarse_op_apply(A, X, L, disp)[0], ref, atol=1e-12)


def test_adjoint_identity_and_hermiticity(rng):
    L = (3, 2, 2, 3)
    disp, _ = stencil(81)
    A = random_general_op(L, 3, 81, rng)
    V = int(np.prod(L))
    u = rng.standard_normal((V, 3, 2)) + 1j * rng.standard_normal((V, 3, 2))
    v = rng.standard_normal((V, 3, 2)) + 1j * rng.standard_normal((V, 3, 2))
    lhs = np.vdot(u, coarse_op_apply(A, v, L, disp))
    rhs = np.vdot(coarse_op_apply_dag(A, u, L, disp), v)
    assert abs(lhs - rhs) < 1e-11 * abs(lhs)
    # generated operators are Hermitian: H = H^dagger
    Ah = coarse_op(L, 3, 81, 5, 2.0)
    assert np.allclose(coarse_op_apply(Ah, v, L, disp), coarse_op_apply_dag(Ah, v, L, disp),
                       atol=1e-12)


def test_native_c_oracle_matches_numpy(rng):
    L = (3, 4, 2, 3)
    for npts in (9, 81):
        disp, _ = stencil(npts)
        A = coarse_op(L, 4, npts, 11, 1.5)
        X = vectors(L, 4, 5, 11)
        ref = coarse_op_apply(A, X, L, disp)
        assert np.allclose(native.coarse_op_apply(A, X, L, disp), ref, rtol=0, atol=1e-12)
        sites = np.array([0, 7, 33, 71])
        ys = native.coarse_op_apply_sites(A[sites], X, L, disp, sites)
        assert np.allclose(ys, ref[sites], rtol=0, atol=1e-12)
        pos = [p for p in range(1, npts) if next(v for v in disp[p] if v != 0) > 0]
        Ahalf = A[:, [0] + pos]
        yh = native.coarse_op_apply_herm_half(Ahalf, X, L, disp[pos])
        assert np.allclose(yh, ref, rtol=0, atol=1e-12)


def test_gram_and_axpy(rng):
    X = rng.standard_normal((40, 3, 5)) + 1j * rng.standard_normal((40, 3, 5))
    Y = rng.standard_normal((40, 3, 4)) + 1j * rng.standard_normal((40, 3, 4))
    G = block_inner(X, Y)
    assert np.allclose(G, np.einsum("nr,ns->rs", np.conj(X.reshape(-1, 5)), Y.reshape(-1, 4)))
    GX = block_inner(X, X)
    assert np.allclose(GX, np.conj(GX.T))
    assert np.min(np.linalg.eigvalsh(GX)) > 0
    M = rng.standard_normal((5, 4)) + 1j * rng.standard_normal((5, 4))
    out = block_axpy(Y, X, M, -0.5)
    assert np.allclose(out.reshape(-1, 4), -0.5 * Y.reshape(-1, 4) + np.einsum(
        "nr,rs->ns", X.reshape(-1, 5), M))
