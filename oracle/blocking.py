"""Block project and promote between fine and coarse degrees of freedom
(Sec. 2.5.1, "Transfer between grids"), complex128.

Test infrastructure only (see the package docstring).

Every coarse site x_c owns a block of v_block fine degrees of freedom and a
basis B(x_c) of n_basis fine vectors restricted to that block.  The two
operations are one small GEMM per coarse site:
    project:  C(x_c) = B(x_c)^dagger F(x_c)    (n_basis x nrhs)
    promote:  F(x_c) = B(x_c) C(x_c)           (v_block x nrhs)
Layouts: basis [n_blocks][v_block][n_basis], fine vectors
[n_blocks][v_block][nrhs], coarse vectors [n_blocks][n_basis][nrhs] (the
coarse layout [V][nb][nrhs] with V = n_blocks, nb = n_basis).
"""
import numpy as np


def block_project(basis, F):
    """C[x] = basis[x]^dagger F[x] for every block x."""
    return np.einsum("xsa,xsr->xar", np.conj(basis), F)


def block_promote(basis, C):
    """F[x] = basis[x] C[x] for every block x."""
    return np.einsum("xsa,xar->xsr", basis, C)
