"""The premise of starting a refinement cycle from kept search blocks, pinned
on the oracle's FP64 BlockCGrQ (Fig. 2 left) with dense linear algebra:

* the search blocks D_k of one run are H-conjugate: D_i^dagger H D_j = 0 for
  i != j (the short block recurrence keeps all earlier directions
  conjugate in exact arithmetic);
* hence sum_k D_k N_k D_k^dagger F with N_k = (D_k^dagger H D_k)^-1 equals the
  Galerkin solution W (W^dagger H W)^-1 W^dagger F over W = [D_1 ... D_m],
  computed here by a dense solve;
* that correction minimises phi(e) = e^dagger H e - 2 Re e^dagger f over the
  span, and phi < 0 = phi(0) for a right-hand side not orthogonal to it (the
  per-column acceptance test of the GPU path).
"""
import numpy as np

from oracle.ops import coarse_op_apply
from oracle.solvers import block_cg_rq
from synth import coarse_op, stencil, vectors

L, NB, NPTS, R = (2, 2, 2, 3), 6, 9, 3


def _problem():
    disp, _ = stencil(NPTS)
    A = coarse_op(L, NB, NPTS, 31, 6.0)
    V = int(np.prod(L))

    def H(X):
        return coarse_op_apply(A, X.reshape(V, NB, -1), L, disp).reshape(V * NB, -1)
    return H, V * NB


def _blocks(H, N, iters=6):
    B = vectors(L, NB, R, 32).reshape(N, R)
    hist = []
    block_cg_rq(lambda X: H(X.reshape(N, -1)).reshape(X.shape), B, tol=1e-14, maxiter=iters,
                history=hist)
    # D used in iteration k (k >= 2) is the D written after iteration k - 1;
    # Z of iteration k is H D_k
    Ds = [hist[k - 2]["D"] for k in range(2, len(hist) + 1)]
    Zs = [hist[k - 1]["Z"] for k in range(2, len(hist) + 1)]
    return Ds, Zs


def test_search_blocks_are_conjugate():
    H, N = _problem()
    Ds, Zs = _blocks(H, N)
    assert len(Ds) >= 4
    for i, Di in enumerate(Ds):
        for j, Zj in enumerate(Zs):
            if i == j:
                continue
            c = np.linalg.norm(Di.conj().T @ Zj)
            assert c <= 1e-9 * np.linalg.norm(Di) * np.linalg.norm(Zj), (i, j, c)
        np.testing.assert_allclose(Zs[i], H(Ds[i]), rtol=0, atol=1e-12 * np.linalg.norm(Zs[i]))


def test_blockwise_sum_equals_galerkin_solution():
    H, N = _problem()
    Ds, Zs = _blocks(H, N)
    rng = np.random.default_rng(5)
    F = rng.standard_normal((N, R)) + 1j * rng.standard_normal((N, R))
    E_sum = np.zeros_like(F)
    for D, Z in zip(Ds, Zs):
        Nk = np.linalg.inv(D.conj().T @ Z)
        E_sum += D @ (Nk @ (D.conj().T @ F))
    W = np.concatenate(Ds, axis=1)
    HW = H(W)
    E_gal = W @ np.linalg.solve(W.conj().T @ HW, W.conj().T @ F)
    assert np.linalg.norm(E_sum - E_gal) <= 1e-9 * np.linalg.norm(E_gal)

    def phi(E):
        HE = H(E)
        return np.real(np.sum(E.conj() * HE, axis=0)) - 2 * np.real(np.sum(E.conj() * F, axis=0))
    p = phi(E_sum)
    assert np.all(p < 0)
    # any other element of the span does no better, column by column
    for _ in range(3):
        d = W @ (rng.standard_normal((W.shape[1], R)) * 1e-2)
        assert np.all(phi(E_sum + d) >= p - 1e-12 * np.abs(p))
    # a plain sum over blocks that are not conjugate is not the Galerkin
    # solution: the premise matters (two copies of one block)
    D0, Z0 = Ds[0], Zs[0]
    Nk = np.linalg.inv(D0.conj().T @ Z0)
    twice = 2 * (D0 @ (Nk @ (D0.conj().T @ F)))
    once = D0 @ (Nk @ (D0.conj().T @ F))
    assert np.all(phi(twice) > phi(once))
