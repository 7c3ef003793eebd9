"""Five-dimensional CG on the GPU against the oracle (oracle.solvers.cg5d):
same iteration count and solution, the DF32 operator variant, duplicated
columns, and the C oracle's true residual on a larger problem."""
import numpy as np
import pytest
import torch

from oracle import native
from oracle.ops import coarse_op_apply
from oracle.solvers import cg5d
from synth import WORKLOADS, coarse_op, load_shift, stencil, vectors

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mrhs():
    assert torch.cuda.is_available()
    import paper_2409_03904_b300 as m
    return m


def test_matches_oracle(mrhs):
    L, nb, npts, R = (3, 2, 2, 3), 8, 81, 5
    disp, _ = stencil(npts)
    A = coarse_op(L, nb, npts, 301, 19.0)
    B = vectors(L, nb, R, 302)
    Xo, io = cg5d(lambda X: coarse_op_apply(A, X, L, disp), B, tol=1e-10, maxiter=500)
    op = mrhs.CoarseOp(torch.from_numpy(A).cuda(), L, disp, ("fp64",))
    X, info = op.solve(torch.from_numpy(B).cuda(), mode="cg5d", tol=1e-10, check_every=1)
    assert info["status"] == 0 and max(info["resid"]) <= 1e-10
    assert info["iters"] == io["iters"]
    assert np.allclose(X.cpu().numpy(), Xo, atol=1e-8 * np.abs(Xo).max())
    Xd, idf = op.solve(torch.from_numpy(B).cuda(), mode="cg5d", tol=1e-10, krylov_prec="df32")
    assert idf["status"] == 0 and max(idf["resid"]) <= 1e-10 and idf["applies"]["df32"] > 0


def test_duplicated_columns(mrhs):
    L, nb, npts = (4, 2, 2, 2), 8, 9
    disp, _ = stencil(npts)
    A = coarse_op(L, nb, npts, 303, 8.0)
    b = vectors(L, nb, 1, 304)
    B = np.concatenate([b, b, 2.0 * b], axis=2)
    op = mrhs.CoarseOp(torch.from_numpy(A).cuda(), L, disp, ("fp64",))
    X, info = op.solve(torch.from_numpy(B).cuda(), mode="cg5d", tol=1e-11)
    Xh = X.cpu().numpy()
    assert np.allclose(Xh[..., 0], Xh[..., 1], atol=1e-13 * np.abs(Xh).max())
    assert np.allclose(Xh[..., 2], 2.0 * Xh[..., 0], atol=1e-10 * np.abs(Xh).max())


def test_workload_true_residual(mrhs):
    w = WORKLOADS["L6_nb16_9pt_r8"]
    disp, _ = stencil(w["npts"])
    A = coarse_op(w["L"], w["nb"], w["npts"], w["seed"], load_shift(w["name"]))
    B = vectors(w["L"], w["nb"], w["nrhs"], w["seed"])
    op = mrhs.CoarseOp(torch.from_numpy(A).cuda(), w["L"], disp, ("fp64",))
    X, info = op.solve(torch.from_numpy(B).cuda(), mode="cg5d", tol=1e-10)
    Xb, ib = op.solve(torch.from_numpy(B).cuda(), mode="fp64", tol=1e-10)
    r = B - native.coarse_op_apply(A, X.cpu().numpy(), w["L"], disp)
    rel = np.linalg.norm(r.reshape(-1, w["nrhs"]), axis=0) / np.linalg.norm(B.reshape(-1, w["nrhs"]), axis=0)
    assert np.max(rel) <= 1.5e-10
    # one Krylov space per column takes at least as many iterations as the block
    assert info["iters"] >= ib["iters"]
