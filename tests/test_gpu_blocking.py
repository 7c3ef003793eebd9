"""Block project / promote on the GPU against the oracle (oracle.blocking):
uneven shapes (ragged right-hand-side chunks, one and many column groups),
FP64 and FP32, the orthonormal round trip, and the size limits."""
import numpy as np
import pytest
import torch

from oracle.blocking import block_project, block_promote

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mrhs():
    assert torch.cuda.is_available()
    import paper_2409_03904_b300 as m
    return m


def rel(Y, ref):
    return float(np.linalg.norm(Y - ref) / np.linalg.norm(ref))


SHAPES = [(37, 48, 8, 5), (64, 256, 64, 12), (5, 7, 3, 33), (9, 100, 256, 16), (3, 300, 64, 64),
          (1, 1, 1, 1)]


@pytest.mark.parametrize("nblk,vb,nbasis,R", SHAPES)
def test_parity(mrhs, nblk, vb, nbasis, R):
    rng = np.random.default_rng(nblk * 1000 + vb + nbasis + R)
    B = rng.standard_normal((nblk, vb, nbasis)) + 1j * rng.standard_normal((nblk, vb, nbasis))
    F = rng.standard_normal((nblk, vb, R)) + 1j * rng.standard_normal((nblk, vb, R))
    C = rng.standard_normal((nblk, nbasis, R)) + 1j * rng.standard_normal((nblk, nbasis, R))
    refC, refF = block_project(B, F), block_promote(B, C)
    for dt, tol in ((torch.complex128, 1e-13), (torch.complex64, 3e-6)):
        Bd, Fd, Cd = (torch.from_numpy(v).to(dt).cuda() for v in (B, F, C))
        assert rel(mrhs.block_project(Bd, Fd).cpu().numpy(), refC) <= tol
        assert rel(mrhs.block_promote(Bd, Cd).cpu().numpy(), refF) <= tol


def test_orthonormal_round_trip(mrhs):
    rng = np.random.default_rng(3)
    nblk, vb, nbasis, R = 16, 64, 24, 12
    B = np.stack([np.linalg.qr(rng.standard_normal((vb, nbasis)) + 1j * rng.standard_normal((vb, nbasis)))[0]
                  for _ in range(nblk)])
    C = rng.standard_normal((nblk, nbasis, R)) + 1j * rng.standard_normal((nblk, nbasis, R))
    Bd, Cd = torch.from_numpy(B).cuda(), torch.from_numpy(C).cuda()
    back = mrhs.block_project(Bd, mrhs.block_promote(Bd, Cd))
    assert rel(back.cpu().numpy(), C) <= 1e-13


def test_limits(mrhs):
    B = torch.zeros((2, 8, 256), dtype=torch.complex128, device="cuda")
    F = torch.zeros((2, 8, 17), dtype=torch.complex128, device="cuda")
    with pytest.raises(mrhs.MrhsError):
        mrhs.block_project(B, F)              # 17 > 16 x (256 / 256)
    assert mrhs.block_project(torch.zeros((0, 8, 4), dtype=torch.complex128, device="cuda"),
                              torch.zeros((0, 8, 2), dtype=torch.complex128, device="cuda")).shape == (0, 4, 2)
