"""GPU autograd: the adjoint kernels against the oracle adjoints and against
central finite differences (h = 1e-6, FP64), on a 6^4 lattice, nb 16,
9-point stencil, 8 RHS, in complex128 and complex64 (the operator)."""
import numpy as np
import pytest
import torch

from oracle.grad import op_vjp, stencil_outer
from oracle.ops import coarse_op_apply
from oracle.solvers import block_cg_rq
from synth import WORKLOADS, STREAM_W, coarse_op, load_shift, stencil, vectors
from tests.test_oracle_grad import hermitian_direction

pytestmark = pytest.mark.gpu
NAME = "L6_nb16_9pt_r8"


@pytest.fixture(scope="module")
def setup():
    assert torch.cuda.is_available()
    import paper_2409_03904_b300 as m
    w = WORKLOADS[NAME]
    disp, _ = stencil(w["npts"])
    A = coarse_op(w["L"], w["nb"], w["npts"], w["seed"], load_shift(NAME))
    B = vectors(w["L"], w["nb"], w["nrhs"], w["seed"])
    W = vectors(w["L"], w["nb"], w["nrhs"], w["seed"], stream=STREAM_W)
    return m, w, disp, A, B, W


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tc32", "fp16x", "fp16"])
def test_operator_gradients(setup, prec):
    """grad X by the adjoint kernel of each precision, grad A by the outer
    product kernel, against the oracle's exact adjoints.  The tensor-core
    forms' grad X carries their quantisation (tested against the quantised
    oracle in test_gpu_ops); against the exact adjoint it meets the same
    bounds as their forward application: 2^-17 (TC32), 2^-9 (FP16X, FP16)."""
    m, w, disp, A, B, W = setup
    dt = torch.complex128 if prec == "fp64" else torch.complex64
    Ad = torch.from_numpy(A).cuda().requires_grad_(True)
    Xd = torch.from_numpy(B).to(dt).cuda().requires_grad_(True)
    Wd = torch.from_numpy(W).to(dt).cuda()
    Y = m.coarse_apply(Ad, Xd, w["L"], disp, prec)
    loss = torch.real(torch.sum(Wd * Y))
    loss.backward()
    GA_ref, GX_ref = op_vjp(A, Xd.detach().cpu().numpy().astype(np.complex128),
                            np.conj(Wd.cpu().numpy().astype(np.complex128)), w["L"], disp)
    tol_x = {"fp64": 1e-12, "fp32": 1e-5, "tc32": 2.0 ** -17, "fp16x": 2.0 ** -9,
             "fp16": 2.0 ** -9}[prec]
    tol_a = 1e-12 if prec == "fp64" else 1e-5
    assert rel(Xd.grad.cpu().numpy(), GX_ref) <= tol_x
    assert rel(Ad.grad.cpu().numpy(), GA_ref) <= tol_a
    assert m.device_error() == 0


def test_operator_gradient_finite_differences(setup):
    m, w, disp, A, B, W = setup
    rng = np.random.default_rng(3)
    Ad = torch.from_numpy(A).cuda().requires_grad_(True)
    Xd = torch.from_numpy(B).cuda().requires_grad_(True)
    Wd = torch.from_numpy(W).cuda()
    loss = torch.real(torch.sum(Wd * m.coarse_apply(Ad, Xd, w["L"], disp)))
    loss.backward()
    f = lambda A_, X_: float(torch.real(torch.sum(Wd * m.coarse_apply(A_, X_, w["L"], disp))))  # noqa
    h = 1e-6
    for _ in range(4):
        dA = torch.from_numpy(rng.standard_normal(A.shape) + 1j * rng.standard_normal(A.shape)).cuda()
        dX = torch.from_numpy(rng.standard_normal(B.shape) + 1j * rng.standard_normal(B.shape)).cuda()
        with torch.no_grad():
            fd = (f(Ad + h * dA, Xd + h * dX) - f(Ad - h * dA, Xd - h * dX)) / (2 * h)
        an = float(torch.real(torch.sum(torch.conj(Ad.grad) * dA) + torch.sum(torch.conj(Xd.grad) * dX)))
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an))


def test_solve_gradients(setup):
    m, w, disp, A, B, W = setup
    L = w["L"]
    opts = dict(tol=1e-13, maxiter=5000)
    Ad = torch.from_numpy(A).cuda().requires_grad_(True)
    Bd = torch.from_numpy(B).cuda().requires_grad_(True)
    Wd = torch.from_numpy(W).cuda()
    X = m.coarse_solve(Ad, Bd, L, disp, **opts)
    loss = torch.real(torch.sum(Wd * X))
    loss.backward()
    # oracle: the same adjoint formulas with the oracle's block CG
    op = lambda V: coarse_op_apply(A, V, L, disp)  # noqa: E731
    Xo, _ = block_cg_rq(op, B, tol=1e-13, maxiter=5000)
    GBo, _ = block_cg_rq(op, np.conj(W), tol=1e-13, maxiter=5000)
    GAo = stencil_outer(GBo, Xo, L, disp, alpha=-1.0)
    assert rel(X.detach().cpu().numpy(), Xo) <= 1e-9
    assert rel(Bd.grad.cpu().numpy(), GBo) <= 1e-9
    assert rel(Ad.grad.cpu().numpy(), GAo) <= 1e-9
    # central finite differences along Hermitian-preserving directions
    rng = np.random.default_rng(11)
    h = 1e-6
    f = lambda A_, B_: float(torch.real(torch.sum(Wd * m.coarse_solve(A_, B_, L, disp, **opts))))  # noqa
    for _ in range(3):
        dA = torch.from_numpy(hermitian_direction(L, w["nb"], w["npts"], rng)).cuda()
        dB = torch.from_numpy(rng.standard_normal(B.shape) + 1j * rng.standard_normal(B.shape)).cuda()
        with torch.no_grad():
            fd = (f(Ad + h * dA, Bd + h * dB) - f(Ad - h * dA, Bd - h * dB)) / (2 * h)
        an = float(torch.real(torch.sum(torch.conj(Ad.grad) * dA) + torch.sum(torch.conj(Bd.grad) * dB)))
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an))


def test_solve_gradients_complex64(setup):
    """The complex64 form of config 3: B, X and grad B in complex64, the
    solve in mixed precision (complex64 tensor-core operators inside, FP64
    outer).  Against the oracle's FP64 adjoints within the complex64
    tolerance 1e-5, and against central finite differences of the FP64
    solve (h = 1e-6) along Hermitian-preserving directions."""
    m, w, disp, A, B, W = setup
    L = w["L"]
    opts = dict(mode="mixed", tol=1e-9, precisions=("fp64", "fp16x", "tc32", "oz"))
    Ad = torch.from_numpy(A).cuda().requires_grad_(True)
    B32 = torch.from_numpy(B).to(torch.complex64).cuda().requires_grad_(True)
    W32 = torch.from_numpy(W).to(torch.complex64).cuda()
    X = m.coarse_solve(Ad, B32, L, disp, **opts)
    assert X.dtype == torch.complex64
    loss = torch.real(torch.sum(W32 * X))
    loss.backward()
    assert B32.grad.dtype == torch.complex64 and Ad.grad.dtype == torch.complex128
    Bh = B32.detach().cpu().numpy().astype(np.complex128)
    Wh = W32.cpu().numpy().astype(np.complex128)
    op = lambda V: coarse_op_apply(A, V, L, disp)  # noqa: E731
    Xo, _ = block_cg_rq(op, Bh, tol=1e-13, maxiter=5000)
    GBo, _ = block_cg_rq(op, np.conj(Wh), tol=1e-13, maxiter=5000)
    GAo = stencil_outer(GBo, Xo, L, disp, alpha=-1.0)
    assert rel(X.detach().cpu().numpy(), Xo) <= 1e-5
    assert rel(B32.grad.cpu().numpy(), GBo) <= 1e-5
    assert rel(Ad.grad.cpu().numpy(), GAo) <= 1e-5
    rng = np.random.default_rng(12)
    h = 1e-6
    Wd = torch.from_numpy(Wh).cuda()
    f64 = dict(tol=1e-13, maxiter=5000)
    f = lambda A_, B_: float(torch.real(torch.sum(Wd * m.coarse_solve(A_, B_, L, disp, **f64))))  # noqa
    B64 = torch.from_numpy(Bh).cuda()
    for _ in range(3):
        dA = torch.from_numpy(hermitian_direction(L, w["nb"], w["npts"], rng)).cuda()
        dB = torch.from_numpy(rng.standard_normal(B.shape) + 1j * rng.standard_normal(B.shape)).cuda()
        with torch.no_grad():
            fd = (f(Ad + h * dA, B64 + h * dB) - f(Ad - h * dA, B64 - h * dB)) / (2 * h)
        gB = B32.grad.to(torch.complex128)
        an = float(torch.real(torch.sum(torch.conj(Ad.grad) * dA) + torch.sum(torch.conj(gB) * dB)))
        assert abs(fd - an) <= 1e-5 * max(1.0, abs(an))
