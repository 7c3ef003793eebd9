"""A seeded gauge-covariant lattice Laplacian, the synthetic fine operator of
the two-level (multigrid) experiments.

The paper's fine operator (domain-wall fermions on gauge ensembles) is not
available.  What a multigrid preconditioner needs from it is a Hermitian
positive operator whose low modes are locally coherent: the covariant
Laplacian
    (H psi)(x) = (8 + m) psi(x) - sum_mu [ U_mu(x) psi(x + mu)
                                           + U_mu(x - mu)^dagger psi(x - mu) ]
on a periodic 4D lattice with nb components per site, whose link matrices
U_mu(x) are random unitaries near the identity, is the standard such model
(the free Laplacian for eps = 0; rougher for larger eps).  Its spectrum lies
in [m, 16 + m].

Random draws and index bookkeeping only: U_mu(x) is the unitary factor Q of
the QR decomposition of 1 + eps G (G standard complex normal from the
counter-based generator at counter (element, site, mu, STREAM_LINK)), with
R's diagonal made positive so that Q is unique.  The result is returned in
the stencil layout A[x][p][a][b] of the 9-point stencil (p = 0 self, then
+e_0, -e_0, +e_1, -e_1, ...), ready for the coarse-operator entry points.
"""
import numpy as np

from .coarse import shifted_sites, stencil, volume
from .philox import complex_normal

STREAM_LINK = 7


def links(L, nb, eps, seed):
    """U[x][mu] (nb x nb unitary) for every site and direction."""
    V = volume(L)
    e = np.arange(nb * nb, dtype=np.int64).reshape(1, 1, nb, nb)
    s = np.arange(V, dtype=np.int64).reshape(V, 1, 1, 1)
    mu = np.arange(4, dtype=np.int64).reshape(1, 4, 1, 1)
    G = complex_normal(e, s, mu, STREAM_LINK, seed)
    M = np.eye(nb)[None, None] + eps * G
    Q, R = np.linalg.qr(M)
    d = np.diagonal(R, axis1=-2, axis2=-1)
    ph = d / np.abs(d)
    return Q * ph[..., None, :]


def covariant_laplacian(L, nb, eps, mass, seed):
    """Coefficients A[x][p][a][b] (complex128, 9-point stencil) of the
    covariant Laplacian above."""
    disp, _ = stencil(9)
    V = volume(L)
    U = links(L, nb, eps, seed)
    A = np.zeros((V, 9, nb, nb), dtype=np.complex128)
    A[:, 0] = (8.0 + mass) * np.eye(nb)
    sites = np.arange(V, dtype=np.int64)
    for p in range(1, 9):
        d = disp[p]
        mu = int(np.nonzero(d)[0][0])
        if d[mu] > 0:
            A[:, p] = -U[:, mu]                       # psi(x + mu) through U_mu(x)
        else:
            back = shifted_sites(L, sites, d)         # x - mu
            A[:, p] = -np.conj(np.swapaxes(U[back, mu], -1, -2))
    return A
