"""Two-level ADEF2 preconditioners and the flexible-vs-stationary outer
solvers (Fig. 1, Fig. 2 right, Sec. 2.3) on the GPU against the oracle.

Inputs (all on the host, none from the CUDA path): a synthetic 9-point fine
operator on 4^4 sites with 4 components, a random block-orthonormal basis
of 6 vectors per 2^4 block, the coarse operator from the oracle's
coarsening, and the lowest eigenpairs of the coarse operator from a dense
eigensolver.  Checked: the transfer (project / promote through the blocked
layout), both preconditioners applied to a block of residuals, the
per-column CG of the variable smoother, flexible ADEF2 with the variable
preconditioner against the oracle's per-column flexible ADEF2, and
Preconditioned BlockCGrQ with the stationary preconditioner against the
oracle's.
"""
import numpy as np
import pytest
import torch

from oracle.blocking import block_project as o_project
from oracle.blocking import block_promote as o_promote
from oracle.coarsen import coarsen_direct, from_blocks, to_blocks
from oracle.deflation import defl_cheby_apply
from oracle.ops import coarse_op_apply
from oracle.solvers import cheby_apply, prec_block_cg_rq
from oracle.twolevel import (adef2_apply, cg_fixed, cg_to_tol, deflated_guess,
                             flex_adef2_columns)
from synth import coarse_op, stencil, vectors
from tests.test_oracle_ops import dense_matrix

pytestmark = pytest.mark.gpu

LF, NBF, BLOCK, NBASIS, NEV, R = (4, 4, 4, 4), 4, (2, 2, 2, 2), 6, 8, 3
SHIFT, LAM_IRS = 6.3, 2.0


def rel_cols(Y, ref):
    R_ = ref.shape[-1]
    d = np.linalg.norm((Y - ref).reshape(-1, R_), axis=0)
    return float(np.max(d / np.linalg.norm(ref.reshape(-1, R_), axis=0)))


@pytest.fixture(scope="module")
def prob():
    assert torch.cuda.is_available()
    import paper_2409_03904_b300 as m
    from paper_2409_03904_b300 import twolevel as tl
    d9, _ = stencil(9)
    d81, _ = stencil(81)
    Af = coarse_op(LF, NBF, 9, 8080, SHIFT)
    As = Af.copy()
    As[:, 0] += LAM_IRS * np.eye(NBF)                       # H + Lambda
    Lc = tuple(l // b for l, b in zip(LF, BLOCK))
    Vc, bv = int(np.prod(Lc)), int(np.prod(BLOCK))
    rng = np.random.default_rng(8081)
    basis = np.empty((Vc, bv * NBF, NBASIS), dtype=np.complex128)
    for k in range(Vc):
        G = rng.standard_normal((bv * NBF, NBASIS)) + 1j * rng.standard_normal((bv * NBF, NBASIS))
        basis[k] = np.linalg.qr(G)[0]
    Hf = lambda V: coarse_op_apply(Af, V, LF, d9)  # noqa: E731
    Ac = coarsen_direct(Hf, LF, NBF, BLOCK, basis, d81)
    ev, W = np.linalg.eigh(dense_matrix(Ac, Lc, d81))
    U = np.ascontiguousarray(W[:, :NEV].reshape(Vc, NBASIS, NEV))
    lam = ev[:NEV]
    hi_f = 1.1 * np.linalg.eigvalsh(dense_matrix(Af, LF, d9))[-1]
    hi_c = 1.1 * ev[-1]
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    fine = m.CoarseOp(dev(Af), LF, d9, ("fp64",))
    shifted = m.CoarseOp(dev(As), LF, d9, ("fp64",))
    coarse = m.CoarseOp(dev(Ac), Lc, d81, ("fp64",))
    T = tl.Transfer(LF, BLOCK, NBF, dev(basis))
    two = tl.TwoLevel(fine, T, coarse)
    B = vectors(LF, NBF, R, 8082)
    return dict(m=m, tl=tl, d9=d9, d81=d81, Af=Af, As=As, Ac=Ac, Lc=Lc, basis=basis, U=U,
                lam=lam, hi_f=hi_f, hi_c=hi_c, fine=fine, shifted=shifted, coarse=coarse, T=T,
                two=two, B=B, dev=dev, Hf=Hf)


def oracle_pieces(p):
    """The oracle's smoothers, coarse solves and Q on [V][nb][R] blocks."""
    d9, d81, Lc = p["d9"], p["d81"], p["Lc"]
    Hf = p["Hf"]
    Hs = lambda V: coarse_op_apply(p["As"], V, LF, d9)  # noqa: E731
    Hc = lambda V: coarse_op_apply(p["Ac"], V, Lc, d81)  # noqa: E731
    proj = lambda F: o_project(p["basis"], to_blocks(F, LF, BLOCK))  # noqa: E731
    prom = lambda C: from_blocks(o_promote(p["basis"], C), LF, BLOCK)  # noqa: E731

    def percol(fn, X):
        out = np.empty_like(X)
        for j in range(X.shape[-1]):
            out[..., j] = fn(X[..., j:j + 1].reshape(-1)).reshape(X.shape[:-1])
        return out

    Um = p["U"].reshape(-1, NEV)

    def one_col(f, shape):
        return lambda v: f(v.reshape(shape + (1,))).reshape(-1)

    cshape = (int(np.prod(Lc)), NBASIS)
    fshape = (int(np.prod(LF)), NBF)
    s_stat = lambda r: cheby_apply(Hf, r, 2.0, p["hi_f"], 8)  # noqa: E731
    c_stat = lambda c: defl_cheby_apply(Hc, p["U"], p["lam"], c, p["lam"][-1] / 10, p["hi_c"],  # noqa
                                        40)
    s_kry = lambda r: percol(lambda v: cg_fixed(one_col(Hs, fshape), v, 7), r)  # noqa: E731

    def c_kry(c):
        return percol(lambda v: cg_to_tol(one_col(Hc, cshape), v,
                                          deflated_guess(Um, p["lam"], v), 4e-2, 500), c)
    return dict(Hf=Hf, proj=proj, prom=prom, s_stat=s_stat, c_stat=c_stat, s_kry=s_kry,
                c_kry=c_kry)


def test_transfer(prob):
    p = prob
    o = oracle_pieces(p)
    C = p["T"].project(p["dev"](p["B"])).cpu().numpy()
    assert rel_cols(C, o["proj"](p["B"])) <= 1e-13
    Cc = vectors(p["Lc"], NBASIS, R, 8083)
    F = p["T"].promote(p["dev"](Cc)).cpu().numpy()
    assert rel_cols(F, o["prom"](Cc)) <= 1e-13


def test_preconditioners(prob):
    p, tl = prob, prob["tl"]
    o = oracle_pieces(p)
    two = p["two"]
    r = p["B"]
    stat = two.stationary((2.0, p["hi_f"], 8),
                          (p["dev"](p["U"]), p["lam"], p["lam"][-1] / 10, p["hi_c"], 40))
    z = stat(p["dev"](r)).cpu().numpy()
    Qs = lambda v: o["prom"](o["c_stat"](o["proj"](v)))  # noqa: E731
    zo = adef2_apply(o["Hf"], o["s_stat"], Qs, r)
    assert rel_cols(z, zo) <= 1e-10
    # the variable one: seven CG steps per column on H + 2, deflated CG to 4e-2
    kry = two.krylov(p["shifted"], 7, p["dev"](p["U"]), p["lam"], 4e-2)
    zk = kry(p["dev"](r)).cpu().numpy()
    Qk = lambda v: o["prom"](o["c_kry"](o["proj"](v)))  # noqa: E731
    zko = adef2_apply(o["Hf"], o["s_kry"], Qk, r)
    assert rel_cols(zk, zko) <= 1e-10
    # the per-column CG alone
    Xs = tl.cg_columns(lambda v: p["shifted"].apply(v, "fp64"), p["dev"](r), iters=7).cpu().numpy()
    assert rel_cols(Xs, o["s_kry"](r)) <= 1e-12


def test_flexible_adef2_with_the_variable_preconditioner(prob):
    p, tl = prob, prob["tl"]
    o = oracle_pieces(p)
    two = p["two"]
    U = p["dev"](p["U"])
    kry = two.krylov(p["shifted"], 7, U, p["lam"], 4e-2)
    Qg = lambda v: two.Q(v, two.deflated_cg_solve(U, p["lam"], 4e-2))  # noqa: E731
    X, info = tl.flex_adef2(two.H, kry, Qg, p["dev"](p["B"]), tol=1e-8, maxiter=200, mmax=1)
    assert info["converged"], info
    fshape = (int(np.prod(LF)), NBF)

    def vec(f):
        return lambda v: f(v.reshape(fshape + (1,))).reshape(-1)
    Qk = lambda v: o["prom"](o["c_kry"](o["proj"](v)))  # noqa: E731
    Mk = lambda v: adef2_apply(o["Hf"], o["s_kry"], Qk, v)  # noqa: E731
    Xo, infos = flex_adef2_columns(vec(o["Hf"]), vec(Mk), vec(Qk), p["B"], tol=1e-8,
                                   maxiter=200, mmax=1)
    for j, io in enumerate(infos):
        assert io["converged"]
        assert abs(info["col_iters"][j] - io["iters"]) <= 1, (j, info["col_iters"], io)
    assert rel_cols(X.cpu().numpy(), Xo) <= 1e-6
    HX = coarse_op_apply(p["Af"], X.cpu().numpy(), LF, p["d9"])
    assert rel_cols(HX, p["B"]) <= 1.5e-8                  # |b_j - H x_j| / |b_j|


def test_prec_block_cg_with_the_stationary_preconditioner(prob):
    p, tl = prob, prob["tl"]
    o = oracle_pieces(p)
    two = p["two"]
    stat = two.stationary((2.0, p["hi_f"], 8),
                          (p["dev"](p["U"]), p["lam"], p["lam"][-1] / 10, p["hi_c"], 40))
    X, info = tl.prec_block_cg(two.H, stat, p["dev"](p["B"]), tol=1e-8, maxiter=200)
    assert info["converged"], info
    Qs = lambda v: o["prom"](o["c_stat"](o["proj"](v)))  # noqa: E731
    Ms = lambda v: adef2_apply(o["Hf"], o["s_stat"], Qs, v)  # noqa: E731
    Xo, io = prec_block_cg_rq(o["Hf"], Ms, p["B"], tol=1e-8, maxiter=200)
    assert io["converged"]
    assert abs(info["iters"] - io["iters"]) <= 1
    assert rel_cols(X.cpu().numpy(), Xo) <= 1e-6
    r = p["B"] - coarse_op_apply(p["Af"], X.cpu().numpy(), LF, p["d9"])
    bn = np.linalg.norm(p["B"].reshape(-1, R), axis=0)
    assert np.max(np.linalg.norm(r.reshape(-1, R), axis=0) / bn) <= 1.5e-8
    assert p["m"].device_error() == 0


def test_zero_right_hand_side_is_rejected(prob):
    p, tl = prob, prob["tl"]
    B = p["B"].copy()
    B[..., 1] = 0
    Bd = p["dev"](B)
    two = p["two"]
    stat = two.stationary((2.0, p["hi_f"], 8),
                          (p["dev"](p["U"]), p["lam"], p["lam"][-1] / 10, p["hi_c"], 40))
    with pytest.raises(ValueError):
        tl.prec_block_cg(two.H, stat, Bd)
    with pytest.raises(ValueError):
        tl.flex_adef2(two.H, stat, lambda v: v, Bd)
    # the per-column CG leaves a zero column at zero
    X = tl.cg_columns(two.H, Bd, tol=1e-8, maxiter=500).cpu().numpy()
    assert np.all(X[..., 1] == 0)
