"""Search blocks kept across the mixed solve's refinement cycles.  Every
inner iteration keeps its search block D and N = (D^dagger H D)^-1; a later
cycle starts from the Galerkin correction over the earlier cycles' blocks
(H-conjugate within a cycle), E_0 = sum_i D_i N_i D_i^dagger F.  The solution
must meet the same tolerance, checked with the C oracle's FP64 residual; the
counters report what was kept and projected; the cap is honoured; with
recycling off nothing is kept."""
import numpy as np
import pytest
import torch

from oracle import native
from synth import BATCH, coarse_op, load_shift, stencil, vectors

pytestmark = pytest.mark.gpu

W = BATCH[10]          # 4^4, nb 24, 81-point stencil, 24 RHS, kappa 1e4


@pytest.fixture(scope="module")
def mrhs():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import paper_2409_03904_b300 as m
    return m


@pytest.fixture(scope="module")
def problem(mrhs):
    disp, _ = stencil(W["npts"])
    A = coarse_op(W["L"], W["nb"], W["npts"], W["seed"], load_shift(W["name"]))
    B = vectors(W["L"], W["nb"], W["nrhs"], W["seed"] + 1)
    op = mrhs.CoarseOp(torch.from_numpy(A).cuda(), W["L"], disp, ("fp64", "fp16x", "tc32", "oz"))
    op.lambda_max("fp16x", 40)
    return op, A, B, disp


def oracle_rel(A, X, B, disp):
    Y = native.coarse_op_apply(A, X, W["L"], disp)
    R = B.shape[-1]
    r = np.linalg.norm((B - Y).reshape(-1, R), axis=0)
    return np.max(r / np.linalg.norm(B.reshape(-1, R), axis=0))


def test_recycled_solve_meets_tol(mrhs, problem):
    op, A, B, disp = problem
    X0, i0 = op.solve(torch.from_numpy(B).cuda(), mode="mixed", tol=1e-8, recycle=0)
    X2, i2 = op.solve(torch.from_numpy(B).cuda(), mode="mixed", tol=1e-8, recycle=2)
    for X, info in ((X0, i0), (X2, i2)):
        assert info["status"] == 0 and max(info["resid"]) <= 1e-8, info
        assert oracle_rel(A, X.cpu().numpy(), B, disp) <= 1.5e-8
    assert i0["recycle_blocks"] == 0 and i0["recycle_projections"] == 0
    assert i2["cycles"] >= 2
    # at most one block per iteration (full-rank iterations only), and two
    # sweeps over the blocks of all earlier cycles at each later cycle start
    assert 0 < i2["recycle_blocks"] <= sum(i2["cycle_iters"])
    kept = np.cumsum(i2["cycle_iters"])
    assert 0 < i2["recycle_projections"] <= 2 * int(np.sum(kept[:-1]))
    print("iterations without / with recycling:", i0["cycle_iters"], i2["cycle_iters"])


def test_recycle_cap_and_single_sweep(mrhs, problem):
    op, A, B, disp = problem
    X, info = op.solve(torch.from_numpy(B).cuda(), mode="mixed", tol=1e-8, recycle=1,
                       recycle_max_blocks=3)
    assert info["status"] == 0 and max(info["resid"]) <= 1e-8
    assert oracle_rel(A, X.cpu().numpy(), B, disp) <= 1.5e-8
    assert 0 < info["recycle_blocks"] <= 3
    assert info["recycle_projections"] <= 3 * (info["cycles"] - 1)


def test_recycle_rejects_negative(mrhs, problem):
    op, A, B, disp = problem
    with pytest.raises(mrhs.MrhsError):
        op.solve(torch.from_numpy(B).cuda(), mode="mixed", recycle=-1)
    with pytest.raises(mrhs.MrhsError):
        op.solve(torch.from_numpy(B).cuda(), mode="mixed", recycle_max_blocks=-2)


def test_recycled_solve_repeatable(mrhs, problem):
    """The kept blocks live on the operator between solves; a second solve
    starts from an empty store and gives the same bits."""
    op, A, B, disp = problem
    Xa, ia = op.solve(torch.from_numpy(B).cuda(), mode="mixed", tol=1e-8, recycle=2)
    Xb, ib = op.solve(torch.from_numpy(B).cuda(), mode="mixed", tol=1e-8, recycle=2)
    assert torch.equal(Xa, Xb)
    assert ia["cycle_iters"] == ib["cycle_iters"] and ia["recycle_blocks"] > 0


def test_recycled_solve_graph_equals_eager(mrhs, problem):
    """The block store runs inside the captured iteration chunks (its slot
    counter lives on the device); replaying the graphs gives the same bits
    as launching every kernel eagerly."""
    op, A, B, disp = problem
    kw = dict(mode="mixed", tol=1e-8, recycle=2, check_every=4)
    Xg, ig = op.solve(torch.from_numpy(B).cuda(), use_graph=1, **kw)
    Xe, ie = op.solve(torch.from_numpy(B).cuda(), use_graph=0, **kw)
    assert torch.equal(Xg, Xe)
    assert ig["cycle_iters"] == ie["cycle_iters"]
    assert ig["recycle_blocks"] == ie["recycle_blocks"] > 0
    assert ig["recycle_projections"] == ie["recycle_projections"] > 0


def test_default_is_plain_restart(mrhs, problem):
    op, A, B, disp = problem
    X, info = op.solve(torch.from_numpy(B).cuda(), mode="mixed", tol=1e-8)
    assert info["recycle_blocks"] == 0 and info["recycle_projections"] == 0


def test_later_cycle_tolerance(mrhs, problem):
    """inner_tol_later loosens only the refinement cycles after the first.
    The first cycle is bit for bit the default one.  The second starts from
    the same state, so with the looser target it stops at the same flag
    read or an earlier one.  The solve still meets tol by the C oracle's
    FP64 residual, and so does a batch.  Tolerances outside their ranges are
    refused."""
    op, A, B, disp = problem
    Bd = torch.from_numpy(B).cuda()
    kw = dict(mode="mixed", tol=1e-8, inner_tol=3e-4, recycle=1, check_every=4)
    X0, i0 = op.solve(Bd, inner_tol_later=0.0, **kw)
    X1, i1 = op.solve(Bd, inner_tol_later=1e-2, **kw)
    for X, info in ((X0, i0), (X1, i1)):
        assert info["status"] == 0 and max(info["resid"]) <= 1e-8, info
        assert oracle_rel(A, X.cpu().numpy(), B, disp) <= 1.5e-8
    assert i0["cycles"] >= 2 and i1["cycles"] >= 2
    assert i1["cycle_iters"][0] == i0["cycle_iters"][0]
    assert i1["cycle_resid"][0] == i0["cycle_resid"][0]
    assert i1["cycle_iters"][1] <= i0["cycle_iters"][1], (i0["cycle_iters"], i1["cycle_iters"])
    print("cycle iterations, later-cycle target 3e-4 / 1e-2:", i0["cycle_iters"], i1["cycle_iters"])
    Xs, infos = mrhs.batch_solve([op], [Bd], tol=1e-8, inner_tol=3e-4, inner_tol_later=1e-2)
    # the library's default for the mixed solve is the later target 1e-2
    Xd, idf = op.solve(Bd, mode="mixed", tol=1e-8, inner_tol=3e-4, recycle=1, check_every=4)
    assert idf["cycle_iters"] == i1["cycle_iters"] and torch.equal(Xd, X1)
    assert infos[0]["status"] == 0 and max(infos[0]["resid"]) <= 1e-8, infos[0]
    assert oracle_rel(A, Xs[0].cpu().numpy(), B, disp) <= 1.5e-8
    for bad in (dict(inner_tol_later=1.0), dict(inner_tol_later=-1e-3), dict(inner_tol=0.0),
                dict(inner_tol=1.5)):
        with pytest.raises(mrhs.MrhsError) as e:
            op.solve(Bd, **{**kw, **bad})
        assert e.value.code == -1, bad
        with pytest.raises(mrhs.MrhsError) as e:
            mrhs.batch_solve([op], [Bd], tol=1e-8, **bad)
        assert e.value.code == -1, bad
