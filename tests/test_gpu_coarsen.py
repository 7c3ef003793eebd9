"""Coarsening on the GPU (momentum-phase method) against the oracle's
definition (oracle.coarsen.coarsen_direct): an 81-point fine operator on
blocks of two directions, identity blocking, a 9-point fine operator on 2^4
blocks with the 9-point coarse stencil, and the coarse operator built from
the result obeying the Galerkin identity on the GPU."""
import numpy as np
import pytest
import torch

from oracle.coarsen import block_maps, coarsen_direct
from oracle.ops import coarse_op_apply
from synth import coarse_op, stencil, vectors

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mrhs():
    assert torch.cuda.is_available()
    import paper_2409_03904_b300 as m
    return m


def orthonormal_basis(rng, Vc, vb, nbasis):
    B = rng.standard_normal((Vc, vb, nbasis)) + 1j * rng.standard_normal((Vc, vb, nbasis))
    return np.ascontiguousarray(np.stack([np.linalg.qr(b)[0] for b in B]))


@pytest.mark.parametrize("block,nbf,nbasis,npts", [((2, 1, 1, 2), 2, 3, 81), ((1, 1, 1, 1), 3, 3, 81),
                                                   ((2, 2, 2, 2), 2, 5, 9)])
def test_against_definition(mrhs, block, nbf, nbasis, npts):
    Lc = (3, 3, 3, 3)
    Lf = tuple(l * b for l, b in zip(Lc, block))
    disp, _ = stencil(npts)
    A = coarse_op(Lf, nbf, npts, 81 + nbf, 6.0)
    Vc, vb = int(np.prod(Lc)), int(np.prod(block)) * nbf
    rng = np.random.default_rng(vb + nbasis)
    if block == (1, 1, 1, 1):
        basis = np.ascontiguousarray(np.broadcast_to(np.eye(nbf, dtype=np.complex128), (Vc, nbf, nbf)))
    else:
        basis = orthonormal_basis(rng, Vc, vb, nbasis)
    ref = coarsen_direct(lambda X: coarse_op_apply(A, X, Lf, disp), Lf, nbf, block, basis, disp)
    op = mrhs.CoarseOp(torch.from_numpy(A).cuda(), Lf, disp, ("fp64",))
    Ac = op.coarsen(block, torch.from_numpy(basis).cuda(), disp).cpu().numpy()
    assert np.abs(Ac - ref).max() <= 1e-12 * np.abs(ref).max()
    if block == (1, 1, 1, 1):
        assert np.abs(Ac - A).max() <= 1e-12 * np.abs(A).max()


def test_galerkin_on_gpu(mrhs):
    """CoarseOp(coarsen(M)) c == P^dagger M P c with the GPU promote / project."""
    Lc, block, nbf, nbasis = (3, 3, 4, 3), (2, 2, 1, 2), 2, 6
    Lf = tuple(l * b for l, b in zip(Lc, block))
    disp, _ = stencil(81)
    A = coarse_op(Lf, nbf, 81, 91, 6.0)
    Vc, vb = int(np.prod(Lc)), int(np.prod(block)) * nbf
    basis = orthonormal_basis(np.random.default_rng(9), Vc, vb, nbasis)
    fine = mrhs.CoarseOp(torch.from_numpy(A).cuda(), Lf, disp, ("fp64",))
    Bd = torch.from_numpy(basis).cuda()
    coarse = mrhs.CoarseOp(fine.coarsen(block, Bd, disp), Lc, disp, ("fp64",))
    C = torch.from_numpy(vectors(Lc, nbasis, 4, 92)).cuda()
    b, i, _ = block_maps(Lf, block)
    bt, it = torch.from_numpy(b).cuda(), torch.from_numpy(i).cuda()
    bv = int(np.prod(block))
    F = mrhs.block_promote(Bd, C).reshape(Vc, bv, nbf, -1)[bt, it]        # blocked -> fine
    MF = fine.apply(F.contiguous(), "fp64")
    Fb = torch.zeros((Vc, bv, nbf, 4), dtype=torch.complex128, device="cuda")
    Fb[bt, it] = MF
    ref = mrhs.block_project(Bd, Fb.reshape(Vc, vb, 4))
    Y = coarse.apply(C, "fp64")
    assert float((Y - ref).abs().max()) <= 1e-12 * float(ref.abs().max())
