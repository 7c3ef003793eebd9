"""GPU parity: every kernel through the C ABI against the FP64 oracle.

Tolerances (relative L2 per right-hand side): FP64 operator 1e-12; FP32 and
BF16/FP16 operators 1e-5 against the oracle's exact value of the same
quantised operator (oracle.lowprec), i.e. what remains is FP32 accumulation.
"""
import numpy as np
import pytest
import torch

from oracle.chol import chol_upper
from oracle.lowprec import lowprec_apply
from oracle.ops import coarse_op_apply, coarse_op_apply_dag
from oracle.solvers import cheby_apply as oracle_cheby
from synth import coarse_op, load_shift, stencil, vectors

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


SHAPES = [((4, 3, 2, 3), 16, 81, 8), ((2, 2, 2, 2), 3, 9, 1), ((3, 3, 3, 3), 24, 9, 4),
          ((1, 1, 1, 1), 8, 81, 2), ((3, 2, 2, 2), 48, 81, 32), ((2, 3, 2, 2), 32, 9, 64),
          ((2, 2, 3, 2), 5, 81, 13), ((2, 2, 2, 3), 64, 81, 64)]


@pytest.mark.parametrize("L,nb,npts,R", SHAPES)
def test_fp64_fp32_op_and_dag(mrhs, L, nb, npts, R):
    disp, _ = stencil(npts)
    rng = np.random.default_rng(nb * 1000 + R)
    V = int(np.prod(L))
    A = rng.standard_normal((V, npts, nb, nb)) + 1j * rng.standard_normal((V, npts, nb, nb))
    X = vectors(L, nb, R, 99)
    op = mrhs.CoarseOp(dev(A), L, disp, ("fp64", "fp32"))
    Y = op.apply(dev(X), "fp64").cpu().numpy()
    assert rel_per_rhs(Y, coarse_op_apply(A, X, L, disp)) <= 1e-12
    Yd = op.apply_dag(dev(X), "fp64").cpu().numpy()
    assert rel_per_rhs(Yd, coarse_op_apply_dag(A, X, L, disp)) <= 1e-12
    Y32 = op.apply(dev(X.astype(np.complex64)), "fp32").cpu().numpy()
    assert rel_per_rhs(Y32, lowprec_apply(A, X, L, disp, "fp32")) <= 1e-5
    Yd32 = op.apply_dag(dev(X.astype(np.complex64)), "fp32").cpu().numpy()
    from oracle.lowprec import quantise_op, quantise_vec
    refd = coarse_op_apply_dag(quantise_op(A, "fp32"), quantise_vec(X, "fp32"), L, disp)
    assert rel_per_rhs(Yd32, refd) <= 1e-5


TC_SHAPES = [((4, 3, 2, 3), 16, 81, 8), ((2, 2, 2, 2), 3, 9, 1), ((3, 3, 3, 3), 24, 9, 4),
             ((3, 2, 2, 2), 48, 81, 32), ((2, 3, 2, 2), 32, 9, 64), ((2, 2, 3, 2), 5, 81, 13),
             ((3, 3, 2, 2), 48, 81, 12), ((2, 2, 2, 2), 64, 9, 16), ((5, 1, 1, 1), 8, 9, 3),
             ((2, 2, 2, 3), 64, 81, 32), ((3, 2, 2, 2), 64, 81, 64), ((2, 2, 2, 2), 63, 9, 31)]


@pytest.mark.parametrize("kind", ["bf16", "fp16", "fp16x", "tc32"])
@pytest.mark.parametrize("L,nb,npts,R", TC_SHAPES)
def test_tensor_core_op(mrhs, kind, L, nb, npts, R):
    disp, _ = stencil(npts)
    A = coarse_op(L, nb, npts, 4242 + nb, 12.0)
    X = vectors(L, nb, R, 4243)
    op = mrhs.CoarseOp(dev(A), L, disp, ("fp64", kind))
    if kind in ("fp16x", "tc32") and R > 32:
        with pytest.raises(mrhs.MrhsError):
            op.apply(dev(X.astype(np.complex64)), kind)
        return
    Y = op.apply(dev(X.astype(np.complex64)), kind).cpu().numpy()
    assert mrhs.device_error() == 0
    ref = lowprec_apply(A, X, L, disp, kind)
    assert rel_per_rhs(Y, ref) <= 1e-5
    # against the unquantised FP64 operator: the quantisation error itself
    exact = coarse_op_apply(A, X, L, disp)
    bound = {"bf16": 2.0 ** -6, "fp16": 2.0 ** -9, "fp16x": 2.0 ** -9, "tc32": 2.0 ** -17}[kind]
    assert rel_per_rhs(Y, exact) <= bound


def test_fp16x_is_linear_and_tc32_is_fp32_class(mrhs):
    L, nb, npts, R = (4, 3, 2, 2), 32, 81, 16
    disp, _ = stencil(npts)
    A = coarse_op(L, nb, npts, 999, 18.0)
    op = mrhs.CoarseOp(dev(A), L, disp, ("fp16", "fp16x", "tc32", "fp32"))
    X1 = dev(vectors(L, nb, R, 1).astype(np.complex64))
    X2 = dev(vectors(L, nb, R, 2).astype(np.complex64))
    def nonlin(kind):
        lhs = op.apply(0.37 * X1 + X2, kind)
        rhs = 0.37 * op.apply(X1, kind) + op.apply(X2, kind)
        return float(torch.linalg.norm(lhs - rhs) / torch.linalg.norm(rhs))
    assert nonlin("fp16x") < 1e-5 < nonlin("fp16")
    exact = coarse_op_apply(A, X1.cpu().numpy().astype(np.complex128), L, disp)
    e32 = rel_per_rhs(op.apply(X1, "tc32").cpu().numpy(), exact)
    ef = rel_per_rhs(op.apply(X1, "fp32").cpu().numpy(), exact)
    assert e32 <= 1e-5 and ef <= 1e-5


@pytest.mark.parametrize("kind", ["bf16", "fp16", "fp16x", "tc32"])
@pytest.mark.parametrize("L,nb,npts,R", [((3, 2, 3, 2), 16, 81, 8), ((3, 2, 2, 2), 48, 81, 32),
                                         ((2, 2, 3, 3), 24, 9, 5)])
def test_tensor_core_dag(mrhs, kind, L, nb, npts, R):
    """The adjoint applications of all four tensor-core forms (a daggered
    packed image built on first use) against the quantised oracle of the
    daggered coefficient field and against the exact FP64 adjoint at the
    forms' analytic bounds."""
    disp, _ = stencil(npts)
    rng = np.random.default_rng(7 + nb)
    V = int(np.prod(L))
    A = rng.standard_normal((V, npts, nb, nb)) + 1j * rng.standard_normal((V, npts, nb, nb))
    X = vectors(L, nb, R, 7)
    op = mrhs.CoarseOp(dev(A), L, disp, ("fp64", kind))
    Y = op.apply_dag(dev(X.astype(np.complex64)), kind).cpu().numpy()
    assert mrhs.device_error() == 0
    # the daggered operator's own coefficient field, quantised by the same rule
    from oracle.ops import neighbour_table
    back = neighbour_table(L, -disp.astype(np.int64))
    Ad = np.empty_like(A)
    for p in range(npts):
        Ad[:, p] = np.conj(np.swapaxes(A[back[p], p], -1, -2))
    ref = lowprec_apply(Ad, X, L, -disp.astype(np.int64), kind)
    assert rel_per_rhs(Y, ref) <= 1e-5
    exact = coarse_op_apply_dag(A, X, L, disp)
    bound = {"bf16": 2.0 ** -6, "fp16": 2.0 ** -9, "fp16x": 2.0 ** -9, "tc32": 2.0 ** -17}[kind]
    assert rel_per_rhs(Y, exact) <= bound


def test_tc_repeat_and_large_nrhs_stream(mrhs):
    """Many sites per CTA (persistent loop, both accumulators, ring wrap)."""
    L, nb, npts, R = (6, 6, 4, 4), 32, 81, 16
    disp, _ = stencil(npts)
    A = coarse_op(L, nb, npts, 5150, 18.0)
    X = vectors(L, nb, R, 5151)
    op = mrhs.CoarseOp(dev(A), L, disp, ("bf16",))
    Xd = dev(X.astype(np.complex64))
    Y1 = op.apply(Xd, "bf16")
    Y2 = op.apply(Xd, "bf16")
    assert torch.equal(Y1, Y2)          # deterministic
    ref = lowprec_apply(A, X, L, disp, "bf16")
    assert rel_per_rhs(Y1.cpu().numpy(), ref) <= 1e-5
    assert mrhs.device_error() == 0


@pytest.mark.parametrize("N,rx,ry", [(1, 1, 1), (1000, 4, 4), (33333, 12, 7), (200000, 32, 32),
                                     (5, 64, 64), (0, 3, 3), (70001, 1, 9), (4097, 16, 3),
                                     (100000, 24, 24), (12345, 64, 1), (777, 9, 64),
                                     (300000, 1, 1)])
def test_block_inner(mrhs, N, rx, ry):
    rng = np.random.default_rng(N + rx)
    X = rng.standard_normal((N, rx)) + 1j * rng.standard_normal((N, rx))
    Y = rng.standard_normal((N, ry)) + 1j * rng.standard_normal((N, ry))
    G = mrhs.block_inner(dev(X), dev(Y)).cpu().numpy()
    ref = np.conj(X).T @ Y
    scale = max(np.linalg.norm(X) * np.linalg.norm(Y), 1e-300)
    assert np.linalg.norm(G - ref) <= 1e-13 * scale
    X32, Y32 = X.astype(np.complex64), Y.astype(np.complex64)
    G32 = mrhs.block_inner(dev(X32), dev(Y32)).cpu().numpy()
    ref32 = np.conj(X32.astype(np.complex128)).T @ Y32.astype(np.complex128)
    assert np.linalg.norm(G32 - ref32) <= 1e-6 * scale
    G2 = mrhs.block_inner(dev(X), dev(Y)).cpu().numpy()
    assert np.array_equal(G, G2)        # fixed reduction order


@pytest.mark.parametrize("N,rin,rout,beta", [(1, 1, 1, 0.0), (1000, 4, 4, 1.0),
                                             (33333, 12, 7, -0.5), (70001, 32, 32, 0.0),
                                             (7, 64, 64, 2.0)])
def test_block_axpy(mrhs, N, rin, rout, beta):
    rng = np.random.default_rng(N + rin)
    X = rng.standard_normal((N, rin)) + 1j * rng.standard_normal((N, rin))
    Y = rng.standard_normal((N, rout)) + 1j * rng.standard_normal((N, rout))
    M = rng.standard_normal((rin, rout)) + 1j * rng.standard_normal((rin, rout))
    ref = beta * Y + X @ M
    out = mrhs.block_axpy(dev(Y), dev(X), dev(M), beta).cpu().numpy()
    assert np.linalg.norm(out - ref) <= 1e-13 * np.linalg.norm(ref)
    out32 = mrhs.block_axpy(dev(Y.astype(np.complex64)), dev(X.astype(np.complex64)), dev(M),
                            beta).cpu().numpy()
    assert np.linalg.norm(out32 - ref) <= 1e-5 * np.linalg.norm(ref)
    if rin == rout:   # in place: X aliases Y
        Xd = dev(X)
        mrhs.block_axpy(Xd, Xd, dev(M), beta)
        ref2 = beta * X + X @ M
        assert np.linalg.norm(Xd.cpu().numpy() - ref2) <= 1e-13 * np.linalg.norm(ref2)


@pytest.mark.parametrize("r", [1, 4, 12, 32, 64])
def test_herm_factor(mrhs, r):
    rng = np.random.default_rng(r)
    T = rng.standard_normal((200, r)) + 1j * rng.standard_normal((200, r))
    G = np.conj(T).T @ T
    S, W, k = mrhs.herm_factor(dev(G))
    S, W = S.cpu().numpy(), W.cpu().numpy()
    assert k == r
    assert np.allclose(S, chol_upper(G), atol=1e-10 * np.sqrt(np.max(np.diag(G).real)))
    assert np.allclose(S @ W, np.eye(r), atol=1e-9)
    if r >= 4:   # rank deficient: duplicated and dependent columns
        T[:, 1] = T[:, 0]
        T[:, 3] = 2 * T[:, 2] - 1j * T[:, 0]
        G = np.conj(T).T @ T
        S, W, k = mrhs.herm_factor(dev(G), 1e-12)
        S, W = S.cpu().numpy(), W.cpu().numpy()
        assert k == r - 2
        Q = T @ W
        assert np.allclose(np.conj(Q).T @ Q, np.diag([1.0] * k + [0.0] * (r - k)), atol=1e-8)
        assert np.allclose(Q @ S, T, atol=1e-8 * np.linalg.norm(T))


@pytest.mark.parametrize("kind", ["fp64", "fp32", "bf16"])
def test_cheby_apply(mrhs, kind):
    L, nb, npts, R = (3, 3, 2, 2), 16, 81, 4
    disp, _ = stencil(npts)
    A = coarse_op(L, nb, npts, 61, 18.0)
    X = vectors(L, nb, R, 62)
    lo, hi, m = 0.5, 40.0, 8
    op = mrhs.CoarseOp(dev(A), L, disp, ("fp64", "fp32", "bf16"))
    if kind == "fp64":
        P = op.cheby(dev(X), lo, hi, m, "fp64").cpu().numpy()
        ref = oracle_cheby(lambda V: coarse_op_apply(A, V, L, disp), X, lo, hi, m)
        assert rel_per_rhs(P, ref) <= 1e-11
    elif kind == "fp32":
        P = op.cheby(dev(X.astype(np.complex64)), lo, hi, m, kind).cpu().numpy()
        ref = oracle_cheby(lambda V: lowprec_apply(A, V, L, disp, kind), X, lo, hi, m)
        assert rel_per_rhs(P, ref) <= 1e-4
    else:
        # every step re-quantises its input to bf16, and a different FP32
        # rounding upstream can flip a code, so the recurrence is compared with
        # the exact polynomial at the quantisation level (2^-8 per step)
        P = op.cheby(dev(X.astype(np.complex64)), lo, hi, m, kind).cpu().numpy()
        ref = oracle_cheby(lambda V: coarse_op_apply(A, V, L, disp), X, lo, hi, m)
        assert rel_per_rhs(P, ref) <= 2e-2


def test_solve_fp64_small(mrhs):
    from tests.test_oracle_ops import dense_matrix
    L, nb, npts, R = (2, 3, 2, 2), 8, 81, 4
    disp, _ = stencil(npts)
    A0 = coarse_op(L, nb, npts, 77, 0.0)
    ev = np.linalg.eigvalsh(dense_matrix(A0, L, disp))
    c = (ev[-1] - 1e3 * ev[0]) / (1e3 - 1)
    A = coarse_op(L, nb, npts, 77, c)
    B = vectors(L, nb, R, 78)
    op = mrhs.CoarseOp(dev(A), L, disp, ("fp64", "fp32", "bf16", "fp16", "fp16x"))
    X, info = op.solve(dev(B), tol=1e-10, maxiter=1000)
    X = X.cpu().numpy()
    H = dense_matrix(A, L, disp)
    ref = np.linalg.solve(H, B.reshape(-1, R))
    assert max(info["resid"]) <= 1e-10
    assert np.linalg.norm(X.reshape(-1, R) - ref) <= 1e3 * 1e-9 * np.linalg.norm(ref)
    res = np.linalg.norm(B.reshape(-1, R) - H @ X.reshape(-1, R), axis=0) / np.linalg.norm(
        B.reshape(-1, R), axis=0)
    assert np.all(res <= 1e-10 * 1.01)
    # preconditioned FP64 and mixed precision reach the same solution
    Xp, ip = op.solve(dev(B), tol=1e-10, precond=1, precond_prec="fp64", cheb_hi=1.1 * ev[-1] + c,
                      cheb_lo=0.1, cheb_order=8)
    assert max(ip["resid"]) <= 1e-10 and ip["iters"] < info["iters"]
    for kind in ("fp16", "bf16", "fp32", "fp16x"):
        Xm, im = op.solve(dev(B), mode="mixed", tol=1e-10, precond=1, precond_prec=kind,
                          cheb_hi=1.1 * ev[-1] + c, cheb_lo=0.2, cheb_order=8)
        assert max(im["resid"]) <= 1e-10, (kind, im)
        assert np.linalg.norm(Xm.cpu().numpy().reshape(-1, R) - ref) <= 1e3 * 1e-9 * np.linalg.norm(ref)
    assert mrhs.device_error() == 0


def test_solve_edge_cases(mrhs):
    L, nb, npts = (2, 2, 2, 2), 4, 9
    disp, _ = stencil(npts)
    A = coarse_op(L, nb, npts, 88, 6.0)
    op = mrhs.CoarseOp(dev(A), L, disp, ("fp64", "fp32", "fp16"))
    B = vectors(L, nb, 4, 89)
    B[:, :, 1] = 0.0                  # zero column
    B[:, :, 3] = B[:, :, 0]           # duplicated column
    for mode, kw in (("fp64", {}), ("mixed", dict(precond=1, precond_prec="fp16", cheb_hi=14.0,
                                                  cheb_lo=0.5, cheb_order=6))):
        X, info = op.solve(dev(B), mode=mode, tol=1e-9, maxiter=500, **kw)
        X = X.cpu().numpy()
        assert np.all(X[:, :, 1] == 0)
        assert max(info["resid"]) <= 1e-9, (mode, info)
        assert np.allclose(X[:, :, 3], X[:, :, 0], atol=1e-8 * np.abs(X).max())
    # single right-hand side and an initial guess that is already the answer
    B1 = B[:, :, :1].copy()
    X1, i1 = op.solve(dev(B1), tol=1e-11)
    X2, i2 = op.solve(dev(B1), X0=X1, tol=1e-9)
    assert i2["iters"] == 0 and max(i2["resid"]) <= 1e-9


def test_solve_refuses_nonfinite_input(mrhs):
    """A NaN or Inf in B, or in a column of X_0 whose B column is not zero,
    is refused before any iteration with MRHS_ERR_NONFINITE (-5) in every
    solve mode and in a batch, instead of being taken for a zero column; the
    operators stay usable."""
    L, nb, npts = (2, 2, 2, 2), 4, 9
    disp, _ = stencil(npts)
    ops = [mrhs.CoarseOp(dev(coarse_op(L, nb, npts, seed, 6.0)), L, disp, ("fp64", "fp16x", "tc32"))
           for seed in (91, 92)]
    op = ops[0]
    B = vectors(L, nb, 4, 93)
    modes = (("fp64", {}), ("mixed", {}), ("cg5d", {}))
    for bad in (np.nan, np.inf):
        Bb = B.copy()
        Bb[3, 1, 2] = bad
        for mode, kw in modes:
            with pytest.raises(mrhs.MrhsError) as e:
                op.solve(dev(Bb), mode=mode, tol=1e-9, maxiter=500, **kw)
            assert e.value.code == -5 and "B column 2" in str(e.value), (mode, str(e.value))
    X0 = np.zeros_like(B)
    X0[0, 0, 1] = np.nan
    for mode, kw in modes:
        with pytest.raises(mrhs.MrhsError) as e:
            op.solve(dev(B), X0=dev(X0), mode=mode, tol=1e-9, maxiter=500, **kw)
        assert e.value.code == -5 and "X0 column 1" in str(e.value), (mode, str(e.value))
    # a NaN guess in a column whose B is zero is cleared: that column's answer is 0
    Bz = B.copy()
    Bz[:, :, 1] = 0.0
    for mode, kw in modes:
        X, info = op.solve(dev(Bz), X0=dev(X0), mode=mode, tol=1e-9, maxiter=500, **kw)
        X = X.cpu().numpy()
        assert np.all(X[:, :, 1] == 0) and np.all(np.isfinite(X)), mode
        assert max(info["resid"]) <= 1e-9, (mode, info)
    # a batch (its interval estimates cached by a first, finite call) names
    # the problem and launches only the column norms; the operators still solve
    Xs, infos = mrhs.batch_solve(ops, [dev(B), dev(B)], tol=1e-8)
    assert all(i["status"] == 0 and max(i["resid"]) <= 1e-8 for i in infos), infos
    Bb = B.copy()
    Bb[5, 2, 0] = np.nan
    n0 = mrhs.launch_count()
    with pytest.raises(mrhs.MrhsError) as e:
        mrhs.batch_solve(ops, [dev(B), dev(Bb)], tol=1e-8)
    assert e.value.code == -5 and "problem 1: B column 0" in str(e.value), str(e.value)
    assert mrhs.launch_count() - n0 <= 8
    Xs, infos = mrhs.batch_solve(ops, [dev(B), dev(B)], tol=1e-8)
    assert all(i["status"] == 0 and max(i["resid"]) <= 1e-8 for i in infos), infos


def test_invalid_arguments(mrhs):
    L, nb, npts = (2, 2, 2, 2), 4, 9
    disp, _ = stencil(npts)
    A = coarse_op(L, nb, npts, 1, 6.0)
    op = mrhs.CoarseOp(dev(A), L, disp, ("fp64",))
    X = dev(vectors(L, nb, 2, 1))
    with pytest.raises(mrhs.MrhsError):
        op.apply(X.to(torch.complex64), "bf16")            # precision not built
    with pytest.raises(mrhs.MrhsError):
        op.apply(X, "fp64", out=X)                         # aliasing
    with pytest.raises(mrhs.MrhsError):
        mrhs.CoarseOp(dev(A), L, np.roll(disp, 1, axis=0), ("fp64",))   # p = 0 not self
    with pytest.raises(TypeError):
        op.apply(X.cpu(), "fp64")


def test_named_workload_solve(mrhs):
    """4^4, nb 24, 9-point, kappa 1e3, 4 RHS, FP64 block CG to 1e-10 against
    the dense 6144 x 6144 LU solve of the same operator."""
    name = "L4_nb24_9pt_r4"
    from synth import WORKLOADS
    w = WORKLOADS[name]
    disp, _ = stencil(w["npts"])
    A = coarse_op(w["L"], w["nb"], w["npts"], w["seed"], load_shift(name))
    B = vectors(w["L"], w["nb"], w["nrhs"], w["seed"])
    op = mrhs.CoarseOp(dev(A), w["L"], disp, ("fp64",))
    X, info = op.solve(dev(B), tol=w["tol"], maxiter=2000)
    assert max(info["resid"]) <= w["tol"]
    from tests.test_oracle_ops import dense_matrix
    H = dense_matrix(A, w["L"], disp)
    ref = np.linalg.solve(H, B.reshape(-1, w["nrhs"]))
    err = np.linalg.norm(X.cpu().numpy().reshape(-1, w["nrhs"]) - ref) / np.linalg.norm(ref)
    assert err <= w["kappa"] * w["tol"]


def test_lambda_max_and_auto_interval(mrhs):
    """Power method below the true maximum and within a few percent; a solve
    with cheb_hi unset uses it (with its margin) and converges."""
    from tests.test_oracle_ops import dense_matrix
    L, nb, npts, R = (3, 2, 2, 2), 8, 81, 3
    disp, _ = stencil(npts)
    A = coarse_op(L, nb, npts, 313, 18.0)
    ev = np.linalg.eigvalsh(dense_matrix(A, L, disp))
    op = mrhs.CoarseOp(dev(A), L, disp, ("fp64", "fp32", "fp16"))
    for prec in ("fp64", "fp32", "fp16"):
        lam = op.lambda_max(prec, 200)
        assert ev[-1] * 0.97 <= lam <= ev[-1] * (1 + 1e-3), (prec, lam, ev[-1])
    B = vectors(L, nb, R, 314)
    X, info = op.solve(dev(B), mode="mixed", tol=1e-9, precond=1, precond_prec="fp16")
    assert max(info["resid"]) <= 1e-9 and info["cheb_hi"] >= ev[-1]


def test_mixed_solve_automatic_precisions(mrhs):
    """With every form built, the mixed solve picks TC32 in the Krylov loop
    and FP16X in the preconditioner up to 32 RHS and FP32 / FP16 above; an
    operator without the split forms falls back to FP32 and FP16 too."""
    L, nb, npts = (3, 2, 2, 2), 8, 81
    disp, _ = stencil(npts)
    A = coarse_op(L, nb, npts, 4321, 18.0)
    full = mrhs.CoarseOp(dev(A), L, disp, ("fp64", "fp32", "fp16", "fp16x", "tc32"))
    plain = mrhs.CoarseOp(dev(A), L, disp, ("fp64", "fp32", "fp16"))
    for op, R, kp, pp in ((full, 8, "tc32", "fp16x"), (full, 40, "fp32", "fp16"),
                          (plain, 12, "fp32", "fp16")):
        B = vectors(L, nb, R, 4322)
        X, info = op.solve(dev(B), mode="mixed", tol=1e-9)
        assert max(info["resid"]) <= 1e-9, info
        assert (info["krylov_prec"], info["precond_prec"]) == (kp, pp)
        assert info["applies"][kp] > 0 and info["applies"][pp] > 0


def test_graph_replay_matches_eager(mrhs):
    """Block-CG chunks captured as CUDA graphs give the same iterates as the
    eager launches (same kernels, same order)."""
    L, nb, npts, R = (4, 3, 2, 3), 16, 81, 8
    disp, _ = stencil(npts)
    A = coarse_op(L, nb, npts, 555, 18.0)
    B = vectors(L, nb, R, 556)
    op = mrhs.CoarseOp(dev(A), L, disp, ("fp64", "fp32", "fp16", "fp16x", "tc32"))
    op.lambda_max("fp16x", 40)      # cached: both solves below reuse it
    for mode in ("fp64", "mixed"):
        kw = dict(mode=mode, tol=1e-9, maxiter=400, check_every=4)
        if mode == "mixed":
            kw.update(precond=1, cheb_order=8)
        n0 = mrhs.launch_count()
        Xg, ig = op.solve(dev(B), use_graph=1, **kw)
        n1 = mrhs.launch_count()
        Xe, ie = op.solve(dev(B), use_graph=0, **kw)
        n2 = mrhs.launch_count()
        assert torch.equal(Xg, Xe), mode
        assert ig["iters"] == ie["iters"] and ig["applies"] == ie["applies"]
        assert n1 - n0 == n2 - n1          # replays are counted as launches
        assert max(ig["resid"]) <= 1e-9


@pytest.mark.parametrize("L,nb,npts,R", [((3, 2, 2, 3), 48, 81, 32), ((4, 3, 2, 3), 16, 9, 8),
                                         ((2, 2, 2, 2), 5, 81, 3), ((3, 3, 2, 2), 24, 81, 64),
                                         ((2, 2, 2, 3), 64, 81, 64)])
def test_df32_operator(mrhs, L, nb, npts, R):
    """Double-float operator against the oracle's FP64 operator and adjoint:
    relative error per RHS well below 1e-11 (2^-44 arithmetic)."""
    disp, _ = stencil(npts)
    rng = np.random.default_rng(nb * 7 + R)
    V = int(np.prod(L))
    A = rng.standard_normal((V, npts, nb, nb)) + 1j * rng.standard_normal((V, npts, nb, nb))
    X = vectors(L, nb, R, 808)
    op = mrhs.CoarseOp(dev(A), L, disp, ("fp64",))
    Y = op.apply(dev(X), "df32").cpu().numpy()
    assert rel_per_rhs(Y, coarse_op_apply(A, X, L, disp)) <= 1e-11
    Yd = op.apply_dag(dev(X), "df32").cpu().numpy()
    assert rel_per_rhs(Yd, coarse_op_apply_dag(A, X, L, disp)) <= 1e-11


def test_df32_cycle_residuals_fp64_confirmation(mrhs):
    """Mixed solve with DF32 cycle residuals (default) and with FP64 ones:
    both end on an FP64 residual <= tol."""
    from synth import WORKLOADS
    w = WORKLOADS["L4_nb24_9pt_r4"]
    L, nb, npts, R = w["L"], w["nb"], w["npts"], w["nrhs"]
    disp, _ = stencil(npts)
    A = coarse_op(L, nb, npts, w["seed"], load_shift(w["name"]))
    B = vectors(L, nb, R, w["seed"])
    op = mrhs.CoarseOp(dev(A), L, disp, ("fp64", "fp16x", "tc32"))
    X1, i1 = op.solve(dev(B), mode="mixed", tol=1e-10)
    X2, i2 = op.solve(dev(B), mode="mixed", tol=1e-10, residual_prec="fp64")
    for X, info in ((X1, i1), (X2, i2)):
        assert info["status"] == 0 and max(info["resid"]) <= 1e-10
        r = B - coarse_op_apply(A, X.cpu().numpy(), L, disp)
        rel = np.linalg.norm(r.reshape(-1, R), axis=0) / np.linalg.norm(B.reshape(-1, R), axis=0)
        assert np.max(rel) <= 1.5e-10
    # one residual per cycle: DF32, or FP64 directly in a cycle whose inner
    # targets are all set by tol; a DF32 residual that meets tol is re-done in FP64
    assert i1["applies"]["df32"] >= 1 and i1["applies"]["fp64"] >= 1
    assert i1["applies"]["df32"] + i1["applies"]["fp64"] >= i1["cycles"]
    assert i1["applies"]["fp64"] <= i1["cycles"]
    assert i2["applies"]["df32"] == 0 and i2["applies"]["fp64"] == i2["cycles"]
