"""Coarsening a fine stencil operator onto a blocked basis (Sec. 2.6,
"Coarse operator"), complex128.

Test infrastructure only (see the package docstring).

The fine operator M acts on a lattice L_f with nb_f components per site and
couples sites at most one step apart in every direction (a stencil inside
{-1,0,1}^4).  The coarse lattice is L_c = L_f / block; coarse site b owns the
fine sites y with floor(y / block) = b, and a basis of n_basis fine vectors
restricted to that block, basis[b][s][k] with s = i * nb_f + a (i the
position of y inside the block, lexicographic with the first direction
fastest, a the fine component).  The coarse matrix elements are
    A_p(b)[j][k] = <phi_j^b | M | phi_k^(b + delta_p)>                 (*)
for every coarse stencil point p.

Two routes: `coarsen_direct` evaluates (*) by applying M to every basis vector
of every block; `coarsen_phase` follows the paper's momentum-phase method,
one application of M per stencil point p to the phased basis
    phi~^p_k = sum_b exp(i b . q^p) phi_k^b,   q^p_mu = 2 pi delta^p_mu / L_c,mu,
block inner products with the basis (a block projection, phase removed),
    T^p(b)[j][k] = exp(-i b . q^p) <phi_j^b | M phi~^p_k> = sum_p' alpha_{p,p'} A_p'(b)[j][k],
    alpha_{p,p'} = exp(i delta^p' . q^p),
and A_p' = sum_p (alpha^-1)_{p',p} T^p.  alpha is invertible when every
coarse extent is at least 3 (so the displacements -1, 0, 1 stay distinct).
"""
import itertools

import numpy as np

from .blocking import block_project, block_promote


def block_maps(Lf, block):
    """(fine site -> coarse block, fine site -> position inside the block)."""
    Lf = np.array(Lf)
    block = np.array(block)
    Lc = Lf // block
    coords = np.array(list(itertools.product(*[range(l) for l in reversed(Lf)])))[:, ::-1]
    bc = coords // block
    ic = coords % block
    b = bc[:, 0] + Lc[0] * (bc[:, 1] + Lc[1] * (bc[:, 2] + Lc[2] * bc[:, 3]))
    i = ic[:, 0] + block[0] * (ic[:, 1] + block[1] * (ic[:, 2] + block[2] * ic[:, 3]))
    return b, i, tuple(int(v) for v in Lc)


def to_blocks(F, Lf, block):
    """Fine vector [V_f][nb_f][R] -> blocked [V_c][v_block][R]."""
    b, i, Lc = block_maps(Lf, block)
    Vc, bv = int(np.prod(Lc)), int(np.prod(block))
    nbf, R = F.shape[1], F.shape[2]
    out = np.zeros((Vc, bv, nbf, R), dtype=np.complex128)
    out[b, i] = F
    return out.reshape(Vc, bv * nbf, R)


def from_blocks(Fb, Lf, block):
    """Blocked [V_c][v_block][R] -> fine [V_f][nb_f][R]."""
    b, i, Lc = block_maps(Lf, block)
    Vc, bv = int(np.prod(Lc)), int(np.prod(block))
    nbf = Fb.shape[1] // bv
    return Fb.reshape(Vc, bv, nbf, Fb.shape[2])[b, i]


def coarse_neighbours(Lc, disp):
    """[npts][V_c]: index of b + delta_p (periodic)."""
    Lc = np.array(Lc)
    coords = np.array(list(itertools.product(*[range(l) for l in reversed(Lc)])))[:, ::-1]
    out = np.empty((len(disp), len(coords)), dtype=np.int64)
    for p, d in enumerate(disp):
        c = (coords + np.asarray(d)) % Lc
        out[p] = c[:, 0] + Lc[0] * (c[:, 1] + Lc[1] * (c[:, 2] + Lc[2] * c[:, 3]))
    return out


def coarsen_direct(apply_M, Lf, nbf, block, basis, disp):
    """A[b][p][j][k] by the definition (*): M applied to the basis vectors of
    every block b' in turn (all n_basis of them as right-hand sides)."""
    Vc, vb, nbasis = basis.shape
    _, _, Lc = block_maps(Lf, block)
    nbr = coarse_neighbours(Lc, disp)
    A = np.zeros((Vc, len(disp), nbasis, nbasis), dtype=np.complex128)
    for bp in range(Vc):
        Pb = np.zeros((Vc, vb, nbasis), dtype=np.complex128)
        Pb[bp] = basis[bp]
        MP = apply_M(from_blocks(Pb, Lf, block))        # [V_f][nb_f][n_basis]
        proj = block_project(basis, to_blocks(MP, Lf, block))   # <phi_j^b | M phi_k^b'>
        for p in range(len(disp)):
            rows = np.nonzero(nbr[p] == bp)[0]          # blocks b with b + delta_p = b'
            A[rows, p] = proj[rows]
    return A


def phase_matrix(Lc, disp):
    """alpha[p][p'] = exp(i delta^p' . q^p), q^p = 2 pi delta^p / L_c."""
    d = np.asarray(disp, dtype=np.float64)
    q = 2.0 * np.pi * d / np.asarray(Lc, dtype=np.float64)
    return np.exp(1j * (q @ d.T))


def coarsen_phase(apply_M, Lf, nbf, block, basis, disp):
    """A[b][p][j][k] by the momentum-phase method: one application of M per
    stencil point, block projections, then alpha^-1 over the stencil index."""
    Vc, vb, nbasis = basis.shape
    _, _, Lc = block_maps(Lf, block)
    coords = np.array(list(itertools.product(*[range(l) for l in reversed(Lc)])))[:, ::-1]
    d = np.asarray(disp, dtype=np.float64)
    q = 2.0 * np.pi * d / np.asarray(Lc, dtype=np.float64)
    T = np.empty((len(disp), Vc, nbasis, nbasis), dtype=np.complex128)
    for p in range(len(disp)):
        ph = np.exp(1j * (coords @ q[p]))               # e^{i b . q^p}
        Phi = from_blocks(basis * ph[:, None, None], Lf, block)
        MPhi = apply_M(Phi)
        T[p] = block_project(basis, to_blocks(MPhi, Lf, block)) * np.conj(ph)[:, None, None]
    ainv = np.linalg.inv(phase_matrix(Lc, disp))
    return np.einsum("qp,pbjk->bqjk", ainv, T)


def galerkin_apply(apply_M, Lf, block, basis, C):
    """P^dagger M P c for coarse vectors C [V_c][n_basis][R]."""
    return block_project(basis, to_blocks(apply_M(from_blocks(block_promote(basis, C), Lf, block)),
                                          Lf, block))
