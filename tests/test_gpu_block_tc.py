"""GPU parity of the tensor-core block algebra (complex64 Gram and block
update, Fig. 2; csrc/blas_tc.cu) against the plain definitions G = X^dagger Y
and Out = beta Y + X M, evaluated in complex128 on the same complex64 inputs.

Bound: each product is formed from exact three-term bf16 splits with the
terms below 2^-23 dropped, and summed in FP32 (over at most 512 rows for the
Gram, then FP64; over the 2 rin reals of a row for the update), so the error
of an entry is a few 2^-23 times the sum of magnitudes of its products:
|G - ref| <= 2e-6 |X|^T |Y| entrywise (the FP32 FMA kernels reach 256 x 2^-24
in the worst case), and the same per element for the update.  The FP32 FMA
kernels (mrhs_block_tc(0)) are checked against the same bound, so the two
paths agree with each other too.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mrhs():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import paper_2409_03904_b300 as m
    prev = m.block_tc(1)
    yield m
    m.block_tc(prev)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def draw(rng, N, r, spread=0.0):
    X = (rng.standard_normal((N, r)) + 1j * rng.standard_normal((N, r))).astype(np.complex64)
    if spread:     # column magnitudes 10^-spread .. 10^spread
        X *= (10.0 ** np.linspace(-spread, spread, r)).astype(np.float32)
    return X


def gram_bound(X, Y):
    ax = np.abs(X.real) + np.abs(X.imag)
    ay = np.abs(Y.real) + np.abs(Y.imag)
    return ax.astype(np.float64).T @ ay.astype(np.float64)


@pytest.mark.parametrize("N,rx,ry,spread", [(1024, 4, 4, 0), (4097, 32, 32, 0),
                                            (65573, 12, 28, 0), (200003, 32, 8, 0),
                                            (130001, 20, 16, 8), (995328, 32, 32, 0)])
def test_gram_tc(mrhs, N, rx, ry, spread):
    rng = np.random.default_rng(N + 7 * rx + ry)
    X, Y = draw(rng, N, rx, spread), draw(rng, N, ry, spread)
    ref = np.conj(X.astype(np.complex128)).T @ Y.astype(np.complex128)
    bound = 2e-6 * gram_bound(X, Y) + 1e-300
    Xd, Yd = dev(X), dev(Y)
    G = mrhs.block_inner(Xd, Yd).cpu().numpy()
    err = np.abs(G.real - ref.real) + np.abs(G.imag - ref.imag)
    assert np.all(err <= bound), float(np.max(err / bound))
    assert np.array_equal(G, mrhs.block_inner(Xd, Yd).cpu().numpy())    # fixed order
    prev = mrhs.block_tc(0)
    try:
        Gs = mrhs.block_inner(Xd, Yd).cpu().numpy()
    finally:
        mrhs.block_tc(prev)
    err_s = np.abs(Gs.real - ref.real) + np.abs(Gs.imag - ref.imag)
    assert np.all(err_s <= bound)
    assert mrhs.device_error() == 0


@pytest.mark.parametrize("N,r", [(1024, 32), (100003, 32), (5000, 16), (333331, 12)])
def test_gram_tc_hermitian(mrhs, N, r):
    """X^dagger X with X passed twice: X's terms serve as both operands."""
    rng = np.random.default_rng(N + r)
    X = draw(rng, N, r)
    Xd = dev(X)
    G = mrhs.block_inner(Xd, Xd).cpu().numpy()
    X128 = X.astype(np.complex128)
    ref = np.conj(X128).T @ X128
    err = np.abs(G.real - ref.real) + np.abs(G.imag - ref.imag)
    assert np.all(err <= 2e-6 * gram_bound(X, X))
    assert np.max(np.abs(np.diag(G).imag)) <= 2e-6 * np.max(np.diag(ref).real)
    Y = dev(X.copy())        # the same values through the general path
    G2 = mrhs.block_inner(Xd, Y).cpu().numpy()
    assert np.all(np.abs(G2 - G) <= 4e-6 * gram_bound(X, X))


@pytest.mark.parametrize("N,rin,rout,beta", [(1024, 4, 4, 1.0), (130001, 32, 32, 0.0),
                                             (33333, 12, 28, -0.5), (12293, 32, 8, 1.0),
                                             (995328, 32, 32, 1.0), (4100, 20, 24, 2.0)])
def test_update_tc(mrhs, N, rin, rout, beta):
    rng = np.random.default_rng(N + rin + 3 * rout)
    X, Y = draw(rng, N, rin), draw(rng, N, rout)
    M = rng.standard_normal((rin, rout)) + 1j * rng.standard_normal((rin, rout))
    M32 = M.astype(np.complex64).astype(np.complex128)
    ref = beta * Y.astype(np.complex128) + X.astype(np.complex128) @ M32
    ax = np.abs(X.real) + np.abs(X.imag)
    am = np.abs(M32.real) + np.abs(M32.imag)
    bound = 2e-6 * (ax.astype(np.float64) @ am + abs(beta) * np.abs(Y)) + 1e-30
    out = mrhs.block_axpy(dev(Y), dev(X), dev(M), beta).cpu().numpy()
    err = np.abs(out.real - ref.real) + np.abs(out.imag - ref.imag)
    assert np.all(err <= bound), float(np.max(err / bound))
    if rin == rout:      # in place: X aliases Y
        Xd = dev(X)
        mrhs.block_axpy(Xd, Xd, dev(M), beta)
        ref2 = beta * X.astype(np.complex128) + X.astype(np.complex128) @ M32
        bound2 = 2e-6 * (ax.astype(np.float64) @ am + abs(beta) * np.abs(X)) + 1e-30
        o2 = Xd.cpu().numpy()
        assert np.all(np.abs(o2.real - ref2.real) + np.abs(o2.imag - ref2.imag) <= bound2)
    prev = mrhs.block_tc(0)
    try:
        outs = mrhs.block_axpy(dev(Y), dev(X), dev(M), beta).cpu().numpy()
    finally:
        mrhs.block_tc(prev)
    err_s = np.abs(outs.real - ref.real) + np.abs(outs.imag - ref.imag)
    assert np.all(err_s <= bound)
    assert mrhs.device_error() == 0


def test_dispatch_edges(mrhs):
    """Shapes beside the tensor-core path (N < 1024, widths not a multiple of
    4) take the FMA kernels and agree with the definition; a view that is not
    16-byte aligned is rejected, as the boundary states."""
    rng = np.random.default_rng(11)
    X = draw(rng, 3001, 33)
    for Xv, Yv in [(X[:1023, :32], X[:1023, :32]), (X[:, :30], X[:, 1:31]), (X[:, :4], X[:, :5])]:
        Xd, Yd = dev(Xv), dev(Yv)
        G = mrhs.block_inner(Xd, Yd).cpu().numpy()
        ref = np.conj(Xv.astype(np.complex128)).T @ Yv.astype(np.complex128)
        assert np.all(np.abs(G - ref) <= 4e-6 * gram_bound(Xv, Yv))
    flat = dev(X.reshape(-1))
    view = flat[1:1 + 2048 * 8].view(2048, 8)        # 8-byte aligned rows
    with pytest.raises(mrhs.MrhsError):
        mrhs.block_inner(view, view)
    assert mrhs.block_tc(1) == 1
    with pytest.raises(Exception):
        mrhs.block_tc(2)


def test_wait_limit_expires_and_recovers(mrhs):
    """The epilogue's bounded wait made to run out on purpose (no fault): the
    kernel records bit 256 (and possibly 64/128/512 of the roles told to
    stop), drains its copies and MMAs, frees its tensor memory and returns;
    with the default limit restored the next call is correct again."""
    lib = mrhs._lib.lib()
    rng = np.random.default_rng(5)
    X = draw(rng, 300000, 32)
    Xd = dev(X)
    M = dev(rng.standard_normal((32, 32)) + 0j)
    assert mrhs.device_error() == 0
    try:
        assert lib.mrhs_debug_wait_limit(1) == 0     # 1 ns: never met by a pipeline
        for call in (lambda: mrhs.block_inner(Xd, Xd), lambda: mrhs.block_axpy(dev(X), Xd, M, 1.0)):
            call()
            err = mrhs.device_error()
            assert err & 256, err
            assert (err & ~(64 | 128 | 256 | 512)) == 0, err
    finally:
        assert lib.mrhs_debug_wait_limit(0) == 0
    G = mrhs.block_inner(Xd, Xd).cpu().numpy()
    assert mrhs.device_error() == 0
    X128 = X.astype(np.complex128)
    assert np.all(np.abs(G - np.conj(X128).T @ X128) <= 2e-6 * gram_bound(X, X))
