"""Small Hermitian factorisations used by block CG (Fig. 2), complex128.

Test infrastructure only (see the package docstring).

The paper writes the factorisation as C^dagger C = G (Fig. 2 right, step 3)
and Q C = R (Fig. 2 left, step 5, a thin QR through Cholesky of R^dagger R).
It does not fix a convention; the reading used here is the unique upper
triangular S with a positive real diagonal.
"""
import numpy as np


class Breakdown(Exception):
    """A Cholesky pivot fell below the relative threshold (rank deficiency)."""


def hermitian_part(G):
    return 0.5 * (G + np.conj(G.T))


def chol_upper(G, tau=1e-14):
    """S upper triangular, real positive diagonal, with S^dagger S = G.

    Textbook column-by-column elimination: for column j
      d = G_jj - sum_{k<j} |S_kj|^2,  S_jj = sqrt(d),
      S_ji = (G_ji - sum_{k<j} conj(S_kj) S_ki) / S_jj   (i > j).
    A pivot d <= tau * max_i G_ii raises Breakdown.
    """
    G = np.asarray(G, dtype=np.complex128)
    n = G.shape[0]
    S = np.zeros((n, n), dtype=np.complex128)
    scale = max(float(np.max(np.real(np.diag(G)))), 0.0) if n else 0.0
    for j in range(n):
        d = float(np.real(G[j, j])) - float(np.sum(np.abs(S[:j, j]) ** 2))
        if not (d > tau * scale) or not np.isfinite(d):
            raise Breakdown(f"pivot {j}: {d!r}")
        s = np.sqrt(d)
        S[j, j] = s
        for i in range(j + 1, n):
            S[j, i] = (G[j, i] - np.sum(np.conj(S[:j, j]) * S[:j, i])) / s
    return S


def upper_inverse(S):
    """Inverse of an upper triangular matrix by back substitution,
    column by column of S^-1 (S W = I)."""
    S = np.asarray(S, dtype=np.complex128)
    n = S.shape[0]
    W = np.zeros((n, n), dtype=np.complex128)
    for j in range(n):
        W[j, j] = 1.0 / S[j, j]
        for i in range(j - 1, -1, -1):
            W[i, j] = -np.sum(S[i, i + 1:j + 1] * W[i + 1:j + 1, j]) / S[i, i]
    return W


def hpd_inverse(G, tau=1e-14):
    """G^-1 for Hermitian positive definite G, as S^-1 S^-dagger."""
    W = upper_inverse(chol_upper(hermitian_part(G), tau))
    return W @ np.conj(W.T)


def pivoted_chol(G, tau=1e-14):
    """Cholesky with complete diagonal pivoting, stopped at numerical rank.

    Returns (S, piv, k): S is k x n upper trapezoidal in the permuted order,
    piv the permutation (S^dagger S = G[piv][:, piv] on the leading block),
    k the number of pivots above tau * max_i G_ii.
    """
    G = np.asarray(G, dtype=np.complex128)
    n = G.shape[0]
    A = G.copy()
    piv = np.arange(n)
    S = np.zeros((n, n), dtype=np.complex128)
    dmax0 = max(float(np.max(np.real(np.diag(G)))), 0.0) if n else 0.0
    k = n
    for j in range(n):
        d = np.array([np.real(A[i, i]) - np.sum(np.abs(S[:j, i]) ** 2) for i in range(j, n)])
        i = j + int(np.argmax(d))
        if not (d[i - j] > tau * dmax0) or not np.isfinite(d[i - j]):
            k = j
            break
        if i != j:
            A[[j, i], :] = A[[i, j], :]
            A[:, [j, i]] = A[:, [i, j]]
            S[:, [j, i]] = S[:, [i, j]]
            piv[[j, i]] = piv[[i, j]]
        s = np.sqrt(d[i - j])
        S[j, j] = s
        for m in range(j + 1, n):
            S[j, m] = (A[j, m] - np.sum(np.conj(S[:j, j]) * S[:j, m])) / s
    return S[:k], piv, k


def block_factor(G, tau=1e-14):
    """Factor a block T with Gram G = T^dagger T (or T^dagger t in the M inner
    product) as T = Q S, Q having orthonormal columns.

    Full rank: S is the upper Cholesky factor and W = S^-1, Q = T W.
    If a pivot falls below tau * max_i G_ii (block rank loss: duplicated or
    dependent right-hand sides, or the block Krylov space running out), the
    factorisation is redone with diagonal pivoting and stopped at rank k:
    S = [S11 S12] P (k x n) and W = P^T [S11^-1; 0] (n x k), so Q = T W keeps
    k columns and the dropped directions (|T u| <= sqrt(tau) |T|) are
    discarded, as in breakdown-free block CG (Ji & Li 2017).
    Returns (S, W).
    """
    Gh = hermitian_part(G)
    try:
        S = chol_upper(Gh, tau)
        return S, upper_inverse(S)
    except Breakdown:
        pass
    Sp, piv, k = pivoted_chol(Gh, tau)
    n = Gh.shape[0]
    S = np.zeros((k, n), dtype=np.complex128)
    S[:, piv] = Sp
    W = np.zeros((n, k), dtype=np.complex128)
    if k:
        W[piv[:k], :] = upper_inverse(Sp[:, :k])
    return S, W
