"""Deflated Chebyshev coarse solve on the GPU against the oracle
(oracle.deflation), with exact eigenvectors of a small operator and with a
random orthonormal deflation basis wider than one 64-column block."""
import numpy as np
import pytest
import torch

from oracle.deflation import defl_cheby_apply
from oracle.ops import coarse_op_apply
from synth import coarse_op, stencil, vectors

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mrhs():
    assert torch.cuda.is_available()
    import paper_2409_03904_b300 as m
    return m


def rel_per_rhs(Y, ref):
    R = ref.shape[-1]
    d = np.linalg.norm((Y - ref).reshape(-1, R), axis=0)
    return float(np.max(d / np.linalg.norm(ref.reshape(-1, R), axis=0)))


def dense(A, L, disp):
    V, npts, nb, _ = A.shape
    N = V * nb
    E = np.eye(N, dtype=np.complex128).reshape(V, nb, N)
    return coarse_op_apply(A, E, L, disp).reshape(N, N)


def test_exact_eigenvectors_fp64_and_df32(mrhs):
    L, nb, npts = (3, 2, 2, 3), 8, 81
    disp, _ = stencil(npts)
    A = coarse_op(L, nb, npts, 77, 19.0)
    lam, W = np.linalg.eigh(dense(A, L, disp))
    assert lam[0] > 0
    V = int(np.prod(L))
    n_ev, lo, hi, order = 20, lam[20] / 2, 1.05 * lam[-1], 40
    U = W[:, :n_ev].reshape(V, nb, n_ev)
    B = vectors(L, nb, 6, 78)
    ref = defl_cheby_apply(lambda X: coarse_op_apply(A, X, L, disp), U, lam[:n_ev], B, lo, hi, order)
    op = mrhs.CoarseOp(torch.from_numpy(A).cuda(), L, disp, ("fp64", "fp16x"))
    Ud = torch.from_numpy(np.ascontiguousarray(U)).cuda()
    for prec, tol in (("fp64", 1e-11), ("df32", 1e-10)):
        X = op.defl_cheby(Ud, lam[:n_ev], torch.from_numpy(B).cuda(), lo, hi, order, prec)
        assert rel_per_rhs(X.cpu().numpy(), ref) <= tol, prec
    # an eigenvector inside the deflation space comes back divided by its eigenvalue
    b = torch.from_numpy(np.ascontiguousarray(W[:, 3:4].reshape(V, nb, 1))).cuda()
    x = op.defl_cheby(Ud, lam[:n_ev], b, lo, hi, order, "fp64").cpu().numpy()
    assert np.allclose(x, W[:, 3:4].reshape(V, nb, 1) / lam[3], atol=1e-12 / lam[3])
    # low precision: the deflation in complex64, the polynomial with FP16X
    X = op.defl_cheby(Ud.to(torch.complex64), lam[:n_ev], torch.from_numpy(B).cuda().to(torch.complex64),
                      lo, hi, order, "fp16x")
    assert rel_per_rhs(X.cpu().numpy(), ref) <= 2e-2


def test_wide_random_basis_and_edge_cases(mrhs):
    """n_ev = 150 (three column blocks, the last ragged) of a random
    orthonormal basis with arbitrary positive values: the GPU follows the
    oracle's formula; n_ev = 0 is the plain polynomial; X may equal B."""
    L, nb, npts = (4, 4, 4, 4), 24, 9
    disp, _ = stencil(npts)
    A = coarse_op(L, nb, npts, 91, 10.0)
    V, N = int(np.prod(L)), int(np.prod(L)) * nb
    rng = np.random.default_rng(5)
    Q, _ = np.linalg.qr(rng.standard_normal((N, 150)) + 1j * rng.standard_normal((N, 150)))
    U = np.ascontiguousarray(Q.reshape(V, nb, 150))
    lam = np.sort(rng.uniform(0.05, 0.5, 150))
    B = vectors(L, nb, 5, 92)
    lo, hi, order = 0.5, 40.0, 16
    apply_H = lambda X: coarse_op_apply(A, X, L, disp)
    ref = defl_cheby_apply(apply_H, U, lam, B, lo, hi, order)
    op = mrhs.CoarseOp(torch.from_numpy(A).cuda(), L, disp, ("fp64",))
    Bd = torch.from_numpy(B).cuda()
    X = op.defl_cheby(torch.from_numpy(U).cuda(), lam, Bd, lo, hi, order, "fp64")
    assert rel_per_rhs(X.cpu().numpy(), ref) <= 1e-11
    X0 = op.defl_cheby(torch.zeros((V, nb, 0), dtype=torch.complex128, device="cuda"), [], Bd,
                       lo, hi, order, "fp64")
    ref0 = defl_cheby_apply(apply_H, U[:, :, :0], lam[:0], B, lo, hi, order)
    assert rel_per_rhs(X0.cpu().numpy(), ref0) <= 1e-11
    Bc = Bd.clone()
    op.defl_cheby(torch.from_numpy(U).cuda(), lam, Bc, lo, hi, order, "fp64", out=Bc)
    assert torch.allclose(Bc, X, rtol=0, atol=1e-13 * float(X.abs().max()))
    with pytest.raises(mrhs.MrhsError):
        op.defl_cheby(torch.from_numpy(U).cuda(), -lam, Bd, lo, hi, order, "fp64")
