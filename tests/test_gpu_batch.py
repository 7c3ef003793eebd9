"""Batched problems: several operators of uneven lattice size, nb, stencil
and nrhs in one persistent tensor-core launch, and side-by-side solves."""
import numpy as np
import pytest
import torch

from oracle import native
from oracle.lowprec import lowprec_apply
from synth import BATCH, coarse_op, load_shift, stencil, vectors

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


SHAPES = [((4, 4, 4, 4), 24, 9, 4), ((4, 3, 2, 3), 32, 81, 8), ((3, 3, 3, 2), 48, 9, 16),
          ((2, 2, 2, 2), 16, 81, 24), ((5, 2, 3, 2), 8, 9, 1)]


@pytest.mark.parametrize("kind", ["fp16", "fp16x", "tc32", "bf16"])
def test_batch_apply_equals_single(mrhs, kind):
    ops, Xs, refs, As, Xh = [], [], [], [], []
    for i, (L, nb, npts, R) in enumerate(SHAPES):
        disp, _ = stencil(npts)
        A = coarse_op(L, nb, npts, 800 + i, 10.0)
        X = vectors(L, nb, R, 900 + i)
        op = mrhs.CoarseOp(torch.from_numpy(A).cuda(), L, disp, (kind,))
        Xd = torch.from_numpy(X.astype(np.complex64)).cuda()
        ops.append(op)
        Xs.append(Xd)
        refs.append(op.apply(Xd, kind))
        As.append(A)
        Xh.append(X)
    Ys = mrhs.batch_apply(ops, Xs, kind)
    torch.cuda.synchronize()
    assert mrhs.device_error() == 0
    for (L, nb, npts, R), Y, ref, A, X in zip(SHAPES, Ys, refs, As, Xh):
        assert torch.equal(Y, ref)            # same per-site MMA order
        disp, _ = stencil(npts)
        exact = lowprec_apply(A, X, L, disp, kind)
        assert rel_per_rhs(Y.cpu().numpy(), exact) <= 1e-5


def oracle_residual(w, A, X, B):
    disp, _ = stencil(w["npts"])
    Y = native.coarse_op_apply(A, X, w["L"], disp)
    r = np.linalg.norm((B - Y).reshape(-1, B.shape[-1]), axis=0)
    return np.max(r / np.linalg.norm(B.reshape(-1, B.shape[-1]), axis=0))


def test_batch_solve_against_oracle(mrhs):
    """Five of the twelve batched problems (host-sized), checked by the C
    oracle's FP64 residual and against one-at-a-time solves."""
    pick = [0, 1, 2, 10, 4]
    ws = [BATCH[i] for i in pick]
    ops, Bs, host = [], [], []
    for w in ws:
        disp, _ = stencil(w["npts"])
        A = coarse_op(w["L"], w["nb"], w["npts"], w["seed"], load_shift(w["name"]))
        B = vectors(w["L"], w["nb"], w["nrhs"], w["seed"])
        ops.append(mrhs.CoarseOp(torch.from_numpy(A).cuda(), w["L"], disp,
                                 ("fp64", "fp32", "fp16", "fp16x", "tc32")))
        Bs.append(torch.from_numpy(B).cuda())
        host.append((A, B))
    n0 = mrhs.launch_count()
    Xs, infos = mrhs.batch_solve(ops, Bs, tol=1e-8)
    for w, X, info, (A, B) in zip(ws, Xs, infos, host):
        assert info["status"] == 0 and max(info["resid"]) <= 1e-8, (w["name"], info)
        assert info["krylov_prec"] == "tc32" and info["precond_prec"] == "fp16x"
        assert oracle_residual(w, A, X.cpu().numpy(), B) <= 1.5e-8
    # one at a time reaches the same tolerance
    for op, B, w in zip(ops, Bs, ws):
        Xi, ii = op.solve(B, mode="mixed", tol=1e-8)
        assert max(ii["resid"]) <= 1e-8
    assert mrhs.launch_count() > n0


def test_full_batch_of_twelve(mrhs):
    """All twelve problems (lattices 4^4..8^4, nb 24..48, 9/81 points, 4..24
    RHS) in one batched solve; the residual of each is checked by the C
    oracle on a sample of sites, against the solve tolerance times the
    column's global |b_j| (|(b - Hx)_S| <= |b - Hx| <= tol |b|)."""
    import synth.device as sdev
    ops, Bs = [], []
    for w in BATCH:
        disp, _ = stencil(w["npts"])
        A = sdev.coarse_op(w["L"], w["nb"], w["npts"], w["seed"], load_shift(w["name"]))
        ops.append(mrhs.CoarseOp(A, w["L"], disp, ("fp64", "fp16x", "tc32")))
        del A
        Bs.append(sdev.vectors(w["L"], w["nb"], w["nrhs"], w["seed"]))
    Xs, infos = mrhs.batch_solve(ops, Bs, tol=1e-8)
    rng = np.random.default_rng(0)
    for w, X, B, info in zip(BATCH, Xs, Bs, infos):
        assert info["status"] == 0 and max(info["resid"]) <= 1e-8, (w["name"], info)
        disp, _ = stencil(w["npts"])
        V = int(np.prod(w["L"]))
        sites = np.sort(rng.choice(V, size=min(24, V), replace=False))
        A_s = coarse_op(w["L"], w["nb"], w["npts"], w["seed"], load_shift(w["name"]), sites=sites)
        Xh, Bh = X.cpu().numpy(), B.cpu().numpy()
        Y = native.coarse_op_apply_sites(A_s, Xh, w["L"], disp, sites)
        r = np.linalg.norm((Bh[sites] - Y).reshape(-1, w["nrhs"]), axis=0)
        bn = np.linalg.norm(Bh.reshape(-1, w["nrhs"]), axis=0)
        assert np.max(r / bn) <= 1.5e-8, w["name"]


def test_autotune_single_and_batch(mrhs):
    """The tuner's candidates agree bit for bit (checked inside the library);
    the cached winner changes the launch, not the result."""
    mrhs.autotune_clear()
    L, nb, npts, R = (4, 4, 4, 4), 32, 81, 16
    disp, _ = stencil(npts)
    A = coarse_op(L, nb, npts, 4321, 18.0)
    op = mrhs.CoarseOp(torch.from_numpy(A).cuda(), L, disp, ("fp16", "tc32"))
    X = torch.from_numpy(vectors(L, nb, R, 4322).astype(np.complex64)).cuda()
    before = op.apply(X, "tc32")
    res = mrhs.autotune(op, "tc32", R, reps=2)
    assert res["candidates"] >= 10 and res["ms"] > 0 and res["ms"] <= res["ms_default"] * 1.5
    assert 0 <= res["pts_per_stage"] <= 12 and res["ctas_per_sm"] in (1, 2)
    assert 2 <= res["max_stages"] <= 32
    assert mrhs.autotune_entries() == 1
    assert torch.equal(op.apply(X, "tc32"), before)
    # a batch is tuned under the list of its members' shapes
    ops, Xs = [op], [X]
    for i, (L2, nb2, npts2, R2) in enumerate(SHAPES[:2]):
        d2, _ = stencil(npts2)
        A2 = coarse_op(L2, nb2, npts2, 990 + i, 10.0)
        ops.append(mrhs.CoarseOp(torch.from_numpy(A2).cuda(), L2, d2, ("fp16",)))
        Xs.append(torch.from_numpy(vectors(L2, nb2, R2, 991 + i).astype(np.complex64)).cuda())
    ref = mrhs.batch_apply(ops, Xs, "fp16")
    res = mrhs.autotune(ops, "fp16", [int(x.shape[2]) for x in Xs], reps=2)
    assert mrhs.autotune_entries() == 2
    for a, b in zip(mrhs.batch_apply(ops, Xs, "fp16"), ref):
        assert torch.equal(a, b)
    assert mrhs.device_error() == 0
    mrhs.autotune_clear()


def test_batch_solve_with_oz_residuals(mrhs):
    """Every problem has the digit-sliced image: the lockstep solve takes its
    cycle residuals from it (one launch per problem, on the problem's own
    stream) and still ends on FP64 residuals <= tol."""
    pick = [0, 2, 10]
    ws = [BATCH[i] for i in pick]
    ops, Bs, host = [], [], []
    for w in ws:
        disp, _ = stencil(w["npts"])
        A = coarse_op(w["L"], w["nb"], w["npts"], w["seed"], load_shift(w["name"]))
        B = vectors(w["L"], w["nb"], w["nrhs"], w["seed"])
        ops.append(mrhs.CoarseOp(torch.from_numpy(A).cuda(), w["L"], disp,
                                 ("fp64", "fp16x", "tc32", "oz")))
        Bs.append(torch.from_numpy(B).cuda())
        host.append((A, B))
    Xs, infos = mrhs.batch_solve(ops, Bs, tol=1e-8)
    for w, X, info, (A, B) in zip(ws, Xs, infos, host):
        assert info["status"] == 0 and max(info["resid"]) <= 1e-8, (w["name"], info)
        assert info["applies"]["oz"] >= 1 and info["applies"]["df32"] == 0, info["applies"]
        assert oracle_residual(w, A, X.cpu().numpy(), B) <= 1.5e-8
    assert mrhs.device_error() == 0
