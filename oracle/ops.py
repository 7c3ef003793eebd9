"""Coarse operator, adjoint, Gram product and block update in complex128.

Test infrastructure only (see the package docstring).

Layouts: coefficients A[x][p][a][b] (site x, stencil point p, row a, column
b); vectors X[x][b][r] (RHS r fastest), equivalently an N x nrhs matrix with
N = V * nb.  Site x = x0 + L0*(x1 + L1*(x2 + L2*x3)), periodic.
"""
import numpy as np


def lattice_volume(L):
    v = 1
    for l in L:
        v *= int(l)
    return v


def neighbour_table(L, disp):
    """nbr[p][x] = index of the site x + delta_p (periodic)."""
    L = [int(l) for l in L]
    V = lattice_volume(L)
    x = np.arange(V, dtype=np.int64)
    c = [x % L[0], (x // L[0]) % L[1], (x // (L[0] * L[1])) % L[2], x // (L[0] * L[1] * L[2])]
    out = np.empty((len(disp), V), dtype=np.int64)
    for p, d in enumerate(disp):
        y = [(c[mu] + int(d[mu])) % L[mu] for mu in range(4)]
        out[p] = y[0] + L[0] * (y[1] + L[1] * (y[2] + L[2] * y[3]))
    return out


def coarse_op_apply(A, X, L, disp):
    """Y(x) = sum_p A_p(x) X(x + delta_p)  (Sec. 2.6, "Applying the coarse
    operator": one batched GEMM per stencil point, batch = coarse volume)."""
    nbr = neighbour_table(L, disp)
    Y = np.zeros(X.shape, dtype=np.complex128)
    for p in range(len(disp)):
        Y += np.matmul(A[:, p], X[nbr[p]])
    return Y


def coarse_op_apply_dag(A, X, L, disp):
    """Adjoint: (H^dagger X)(x) = sum_p A_p(x - delta_p)^dagger X(x - delta_p).

    From H[x, x+delta_p] = A_p(x): H^dagger[y, x] = A_p(x)^dagger with
    y = x + delta_p, i.e. the row y collects A_p(y - delta_p)^dagger.
    """
    minus = -np.asarray(disp, dtype=np.int64)
    back = neighbour_table(L, minus)          # x - delta_p
    Y = np.zeros(X.shape, dtype=np.complex128)
    for p in range(len(disp)):
        src = back[p]
        Y += np.matmul(np.conj(np.swapaxes(A[src, p], -1, -2)), X[src])
    return Y


def as_matrix(X):
    """[V][nb][nrhs] -> [N][nrhs] view."""
    return X.reshape(-1, X.shape[-1])


def block_inner(X, Y):
    """Gram product G = X^dagger Y  (nrhs_x x nrhs_y), the block inner
    product of Fig. 2 (D^dagger Z, T^dagger t, ...)."""
    return np.conj(as_matrix(X)).T @ as_matrix(Y)


def block_axpy(Y, X, M, beta):
    """beta * Y + X M with M (nrhs_in x nrhs_out): the block rotations and
    updates of Fig. 2 (X + D M, Q - Z M, D S^dagger, ...)."""
    out = as_matrix(X) @ M
    if beta != 0.0:
        out = out + beta * as_matrix(Y)
    return out.reshape(X.shape[:-1] + (M.shape[1],))


def column_norms(X):
    return np.sqrt(np.sum(np.abs(as_matrix(X)) ** 2, axis=0))
