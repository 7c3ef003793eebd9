"""Adjoints (vector-Jacobian products) of the coarse operator and of the solve.

Test infrastructure only (see the package docstring).

Convention (the one torch uses for complex tensors): for a real loss L and a
complex tensor z, grad z = dL/dRe z + i dL/dIm z, so dL = Re sum conj(grad z) dz.
Each coefficient A_p(x)[a][b] is an independent complex parameter.

* Operator Y = H X, Y(x) = sum_p A_p(x) X(x + delta_p):
      grad X = H^dagger grad Y,
      grad A_p(x) = grad Y(x) X(x + delta_p)^dagger   (sum over RHS columns).
* Solve X = H^-1 B (H Hermitian, as block CG requires):
      grad B = H^-dagger grad X = H^-1 grad X,
      grad A_p(x) = -grad B(x) X(x + delta_p)^dagger.
These follow from dY = dA X + A dX and dX = H^-1 (dB - dH X).
"""
import numpy as np

from .ops import coarse_op_apply_dag, neighbour_table


def stencil_outer(G, X, L, disp, alpha=1.0):
    """alpha * G(x) X(x + delta_p)^dagger for every site and stencil point:
    [V][npts][nb][nb]."""
    nbr = neighbour_table(L, disp)
    out = np.empty((G.shape[0], len(disp), G.shape[1], X.shape[1]), dtype=np.complex128)
    for p in range(len(disp)):
        out[:, p] = np.matmul(G, np.conj(np.swapaxes(X[nbr[p]], -1, -2)))
    return alpha * out


def op_vjp(A, X, GY, L, disp):
    """(grad A, grad X) of Y = H X given grad Y."""
    return stencil_outer(GY, X, L, disp), coarse_op_apply_dag(A, GY, L, disp)


def solve_vjp(solve, X, GX, L, disp):
    """(grad A, grad B) of X = H^-1 B given grad X; `solve` applies H^-1
    (H Hermitian, so H^-dagger = H^-1)."""
    GB = solve(GX)
    return stencil_outer(GB, X, L, disp, alpha=-1.0), GB
