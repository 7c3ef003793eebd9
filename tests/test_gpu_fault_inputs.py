"""Host-side fault injection in the solves; no GPU fault is made.

Three faults are planted on a 2^4 lattice, nb 4, 9-point stencil, 4 RHS:
- an iteration cap too small to converge;
- a coefficient field holding a NaN;
- an operator whose hop pairs are not Hermitian, fed to block CG (Fig. 2
  assumes H Hermitian positive definite).

In every solve mode each call must:
- return promptly with a status code;
- write X and info where the header says so;
- leave the library usable for the next solve.
"""
import time

import numpy as np
import pytest
import torch

from synth import coarse_op, stencil, vectors

pytestmark = pytest.mark.gpu

L, NB, NPTS, R = (2, 2, 2, 2), 4, 9, 4
MODES = ("fp64", "mixed", "cg5d")


@pytest.fixture(scope="module")
def mrhs():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import paper_2409_03904_b300 as m
    return m


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def make_op(mrhs, A):
    disp, _ = stencil(NPTS)
    return mrhs.CoarseOp(dev(A), L, disp, ("fp64", "fp16x", "tc32"))


def colnorms(Z):
    return np.linalg.norm(Z.reshape(-1, Z.shape[-1]), axis=0)


def test_iteration_cap_reports_the_last_iterate(mrhs):
    """maxiter = 2 cannot reach 1e-12. The status is NOT_CONVERGED, the
    reported residuals are those of the X returned, and the default call
    raises with the same code."""
    op = make_op(mrhs, coarse_op(L, NB, NPTS, 71, 6.0))
    B = dev(vectors(L, NB, R, 72))
    Bh = B.cpu().numpy()
    for mode in MODES:
        X, info = op.solve(B, mode=mode, tol=1e-12, maxiter=2, raise_on_fail=False)
        assert info["status"] == -3 and 1 <= info["iters"] <= 2, (mode, info)
        Xh = X.cpu().numpy()
        assert np.all(np.isfinite(Xh)), mode
        true = colnorms(Bh - op.apply(X, "fp64").cpu().numpy()) / colnorms(Bh)
        rep = np.asarray(info["resid"][:R])
        assert np.max(rep) > 1e-12, (mode, rep)
        assert np.allclose(rep, true, rtol=1e-6, atol=1e-14), (mode, rep, true)
        with pytest.raises(mrhs.MrhsError) as e:
            op.solve(B, mode=mode, tol=1e-12, maxiter=2)
        assert e.value.code == -3, mode


def test_nan_coefficient_is_reported(mrhs):
    """One NaN in the coefficient field (site 3, stencil point 1) makes
    every solve mode end with BREAKDOWN (a NaN pivot) or NONFINITE, well
    within its iteration cap. An operator without the NaN then solves
    normally."""
    A = coarse_op(L, NB, NPTS, 73, 6.0)
    A[3, 1, 2, 0] = np.nan
    bad = make_op(mrhs, A)
    B = dev(vectors(L, NB, R, 74))
    for mode in MODES:
        t0 = time.time()
        with pytest.raises(mrhs.MrhsError) as e:
            bad.solve(B, mode=mode, tol=1e-9, maxiter=200)
        assert e.value.code in (-4, -5), (mode, str(e.value))
        assert time.time() - t0 < 60, mode
    assert mrhs.device_error() == 0
    good = make_op(mrhs, coarse_op(L, NB, NPTS, 73, 6.0))
    for mode in MODES:
        X, info = good.solve(B, mode=mode, tol=1e-9, maxiter=500)
        assert info["status"] == 0 and max(info["resid"]) <= 1e-9, (mode, info)


def test_non_hermitian_operator_returns_a_status(mrhs):
    """The +x hops scaled by 1.5 and their partners left as they were: H is
    no longer Hermitian. Block CG then has no guarantee. Each mode must
    still return within its cap with a status code: converged,
    NOT_CONVERGED or BREAKDOWN. On NOT_CONVERGED the X returned is finite
    and its residual is the one reported."""
    disp, _ = stencil(NPTS)
    A = coarse_op(L, NB, NPTS, 75, 6.0)
    p = next(i for i in range(NPTS) if tuple(disp[i]) == (1, 0, 0, 0))
    A[:, p] *= 1.5
    op = make_op(mrhs, A)
    B = dev(vectors(L, NB, R, 76))
    Bh = B.cpu().numpy()
    for mode in MODES:
        t0 = time.time()
        try:
            X, info = op.solve(B, mode=mode, tol=1e-9, maxiter=100, raise_on_fail=False)
            code = info["status"]
        except mrhs.MrhsError as e:
            X, code = None, e.code
        assert code in (0, -3, -4), (mode, code)
        assert time.time() - t0 < 60, mode
        if code == -3:
            Xh = X.cpu().numpy()
            assert np.all(np.isfinite(Xh)), mode
            true = colnorms(Bh - op.apply(X, "fp64").cpu().numpy()) / colnorms(Bh)
            assert np.allclose(np.asarray(info["resid"][:R]), true, rtol=1e-6, atol=1e-14), mode
    assert mrhs.device_error() == 0
