"""GPU parity of the tensor-core block project / promote (Sec. 2.5.1;
csrc/blocking_tc.cu) against their definitions C(x) = B(x)^dagger F(x) and
F(x) = B(x) C(x), evaluated in complex128 on the same complex64 inputs.

Bound: products from exact three-term bf16 splits with the terms below 2^-23
dropped, summed in FP32 tensor memory over the contraction (v_block fine
rows, or 2 n_basis reals), so an entry is within a few 2^-23 of the sum of
magnitudes of its products (2e-6 |B|^T |F| entrywise, as for the Gram);
checked also against the FP32 FMA kernels (mrhs_block_tc(0)), which meet the
same bound.  Shapes on the tensor-core path: v_block a multiple of 64,
n_basis a multiple of 8 up to 64, nrhs a multiple of 4 up to 32.
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


def draw(rng, shape):
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(np.complex64)


def absum(z):
    return (np.abs(z.real) + np.abs(z.imag)).astype(np.float64)


def err(a, b):
    return np.abs(a.real - b.real) + np.abs(a.imag - b.imag)


SHAPES = [(64, 256, 64, 12), (7, 64, 8, 4), (33, 128, 24, 32), (300, 192, 40, 20),
          (1, 64, 64, 32), (4096, 256, 64, 12)]


@pytest.mark.parametrize("nblk,vb,nbasis,R", SHAPES)
def test_project_promote_tc(mrhs, nblk, vb, nbasis, R):
    rng = np.random.default_rng(nblk + vb + nbasis + R)
    B, F, C = draw(rng, (nblk, vb, nbasis)), draw(rng, (nblk, vb, R)), draw(rng, (nblk, nbasis, R))
    B128, F128, C128 = (v.astype(np.complex128) for v in (B, F, C))
    refC = np.matmul(np.conj(B128).transpose(0, 2, 1), F128)
    refF = np.matmul(B128, C128)
    boundC = 2e-6 * np.matmul(absum(B).transpose(0, 2, 1), absum(F)) + 1e-30
    boundF = 2e-6 * np.matmul(absum(B), absum(C)) + 1e-30
    Bd, Fd, Cd = (torch.from_numpy(v).cuda() for v in (B, F, C))
    outs = {}
    for mode in (1, 0):
        prev = mrhs.block_tc(mode)
        try:
            gC = mrhs.block_project(Bd, Fd).cpu().numpy()
            gF = mrhs.block_promote(Bd, Cd).cpu().numpy()
        finally:
            mrhs.block_tc(prev)
        assert np.all(err(gC, refC) <= boundC), (mode, float(np.max(err(gC, refC) / boundC)))
        assert np.all(err(gF, refF) <= boundF), (mode, float(np.max(err(gF, refF) / boundF)))
        outs[mode] = (gC, gF)
    # the tensor-core results are deterministic
    assert np.array_equal(mrhs.block_project(Bd, Fd).cpu().numpy(), outs[1][0])
    assert np.array_equal(mrhs.block_promote(Bd, Cd).cpu().numpy(), outs[1][1])
    assert mrhs.device_error() == 0


def test_orthonormal_round_trip_tc(mrhs):
    """project(promote(C)) = C for an orthonormal basis, to FP32 accuracy."""
    rng = np.random.default_rng(5)
    nblk, vb, nbasis, R = 40, 128, 32, 12
    B = np.stack([np.linalg.qr(rng.standard_normal((vb, nbasis)) +
                               1j * rng.standard_normal((vb, nbasis)))[0] for _ in range(nblk)])
    B = B.astype(np.complex64)
    C = draw(rng, (nblk, nbasis, R))
    Bd, Cd = torch.from_numpy(B).cuda(), torch.from_numpy(C).cuda()
    back = mrhs.block_project(Bd, mrhs.block_promote(Bd, Cd)).cpu().numpy()
    assert np.linalg.norm(back - C) <= 1e-5 * np.linalg.norm(C)
