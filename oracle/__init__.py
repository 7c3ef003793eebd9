"""FP64 CPU oracle for the multi-RHS coarse operator and block CG.

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
baseline leg of the benchmark may import, call, link or run anything in this
package; the product path (the CUDA library and its Python binding) never
does, and shares no code with it.  The seeded input generators in ``synth``
are the one thing both sides use.

Every function is a plain restatement of the paper (P. Boyle, "Multiple right
hand side multigrid for domain wall fermions with a multigrid preconditioned
block conjugate gradient algorithm", arXiv:2409.03904), in complex128:

* ``ops``      coarse operator Y(x) = sum_p A_p(x) X(x+delta_p)   (Sec. 2.6,
               "Applying the coarse operator"), its adjoint, the Gram product
               X^dagger Y and the block update beta Y + X M (Fig. 2).
* ``chol``     upper Cholesky S^dagger S = G and triangular inverse (Fig. 2).
* ``solvers``  BlockCGrQ (Fig. 2 left), Preconditioned BlockCGrQ (Fig. 2
               right), the Chebyshev approximation to 1/x used as a static
               preconditioner (Sec. 2.3), plain CG, the power method, Lanczos
               extreme-eigenvalue estimates, defect correction.
* ``lowprec``  the quantised operators that the BF16 / FP16 / FP32 GPU paths
               evaluate exactly (up to FP32 accumulation order).
* ``grad``     adjoints of the operator and of the solve.
* ``native``   the same coarse operator as plain C loops (OpenMP), used
               where numpy is too slow (large lattices, CPU baseline).

Parity pins live in tests/test_oracle_*.py: dense assembled matrices with a
LAPACK solve, momentum-space closed forms, the free lattice Laplacian,
adjoint/Hermiticity identities, block CG with one RHS against plain CG,
finite termination, the Chebyshev residual closed form, and finite
differences for the gradients.
"""
