"""Hermitian pairing of the tensor-core kernels: for an exactly Hermitian
operator (A_q(x + delta_p) = A_p(x)^dagger, q the partner of p) with nb a
multiple of 16, the opt-in pairing reads one coefficient tile per point pair and uses it twice,
the second time transposed and conjugated.  The paired and the unpaired
kernels must agree to FP32 summation order, and both must match the oracle's
quantised operator (1e-5 relative, as the other tensor-core tests)."""
import numpy as np
import pytest
import torch

from oracle.lowprec import lowprec_apply
from oracle.ops import coarse_op_apply
from synth import coarse_op, stencil, vectors

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mrhs():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import paper_2409_03904_b300 as m
    return m


def rel_per_rhs(Y, ref):
    Y = np.asarray(Y).reshape(-1, ref.shape[-1])
    ref = ref.reshape(-1, ref.shape[-1])
    num = np.linalg.norm(Y - ref, axis=0)
    den = np.maximum(np.linalg.norm(ref, axis=0), 1e-300)
    return np.max(num / den)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


SHAPES = [((4, 4, 4, 4), 16, 81, 8), ((3, 2, 5, 4), 48, 81, 32), ((2, 2, 2, 2), 64, 9, 16),
          ((6, 3, 2, 2), 32, 9, 1), ((4, 3, 2, 3), 48, 81, 12), ((1, 1, 1, 1), 16, 81, 4)]


@pytest.mark.parametrize("kind", ["fp16", "fp16x", "tc32", "bf16"])
@pytest.mark.parametrize("L,nb,npts,R", SHAPES)
def test_paired_equals_unpaired_and_oracle(mrhs, kind, L, nb, npts, R):
    disp, _ = stencil(npts)
    A = coarse_op(L, nb, npts, 9090 + nb, 12.0)
    X = vectors(L, nb, R, 9091).astype(np.complex64)
    op = mrhs.CoarseOp(dev(A), L, disp, ("fp64", kind))
    assert op.hermitian() == 0                  # opt-in
    assert op.hermitian(1) == 1
    Yp = op.apply(dev(X), kind).cpu().numpy()
    Ypd = op.apply_dag(dev(X), kind).cpu().numpy()     # H^dagger = H: the same kernel
    assert op.hermitian(0) == 0
    Yu = op.apply(dev(X), kind).cpu().numpy()
    ref = lowprec_apply(A, X.astype(np.complex128), L, disp, kind)
    assert rel_per_rhs(Yp, Yu) <= 2e-6
    assert rel_per_rhs(Yp, ref) <= 1e-5
    assert rel_per_rhs(Yu, ref) <= 1e-5
    assert np.array_equal(Yp, Ypd)
    assert op.hermitian(2) == 2
    assert mrhs.device_error() == 0


def test_non_hermitian_operator_is_not_paired(mrhs):
    L, nb, npts = (2, 2, 2, 2), 16, 9
    disp, _ = stencil(npts)
    rng = np.random.default_rng(3)
    V = int(np.prod(L))
    A = rng.standard_normal((V, npts, nb, nb)) + 1j * rng.standard_normal((V, npts, nb, nb))
    op = mrhs.CoarseOp(dev(A), L, disp, ("fp64", "fp16"))
    assert op.hermitian() == 0
    with pytest.raises(mrhs.MrhsError):
        op.hermitian(1)
    X = vectors(L, nb, 4, 5).astype(np.complex64)
    Y = op.apply(dev(X), "fp16").cpu().numpy()
    assert rel_per_rhs(Y, lowprec_apply(A, X.astype(np.complex128), L, disp, "fp16")) <= 1e-5


def test_batch_with_paired_and_unpaired_problems(mrhs):
    """One persistent launch over a Hermitian nb-48 problem (paired), a
    Hermitian nb-24 one (not a multiple of 16: unpaired) and a paired nb-16
    one equals the single launches bit for bit."""
    specs = [((3, 2, 2, 2), 48, 81, 8), ((2, 2, 2, 2), 24, 9, 4), ((4, 2, 2, 2), 16, 81, 12)]
    ops, Xs, singles = [], [], []
    for i, (L, nb, npts, R) in enumerate(specs):
        disp, _ = stencil(npts)
        A = coarse_op(L, nb, npts, 700 + i, 12.0)
        op = mrhs.CoarseOp(dev(A), L, disp, ("fp64", "fp16x"))
        op.hermitian(1)                         # nb 24 is paired in the kernel only if nb % 16 == 0
        X = dev(vectors(L, nb, R, 710 + i).astype(np.complex64))
        ops.append(op)
        Xs.append(X)
        singles.append(op.apply(X, "fp16x"))
    Ys = mrhs.batch_apply(ops, Xs, "fp16x")
    for Y, Y1 in zip(Ys, singles):
        assert torch.equal(Y, Y1)


def test_paired_solve_matches_fp64_oracle(mrhs):
    L, nb, npts, R = (4, 4, 3, 3), 32, 81, 8
    disp, _ = stencil(npts)
    A = coarse_op(L, nb, npts, 4411, 18.0)
    B = vectors(L, nb, R, 4412)
    op = mrhs.CoarseOp(dev(A), L, disp, ("fp64", "fp16x", "tc32"))
    assert op.hermitian(1) == 1
    X, info = op.solve(dev(B), mode="mixed", tol=1e-9)
    assert info["status"] == 0 and max(info["resid"]) <= 1e-9
    r = B - coarse_op_apply(A, X.cpu().numpy(), L, disp)
    rel = np.linalg.norm(r.reshape(-1, R), axis=0) / np.linalg.norm(B.reshape(-1, R), axis=0)
    assert np.max(rel) <= 1.5e-9
