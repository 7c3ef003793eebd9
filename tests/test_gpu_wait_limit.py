"""The bounded waits of the tensor-core kernels, made to run out on purpose
(no GPU fault involved): with the epilogue's accumulator wait limited to a
microsecond, an application of the FP16 (op_tc.cu) and of the digit-sliced
(op_oz.cu) kernel records its bit in mrhs_device_error, drains its copies and
MMAs, frees its tensor memory and returns; the context stays usable, and with
the default limit restored the next application is correct again."""
import numpy as np
import pytest
import torch

from oracle.lowprec import lowprec_apply
from oracle.ops import coarse_op_apply
from synth import coarse_op, stencil, vectors

pytestmark = pytest.mark.gpu


def rel(Y, ref):
    return float(np.linalg.norm(Y - ref) / np.linalg.norm(ref))


@pytest.mark.parametrize("prec,bit,mask", [("fp16", 4, 7), ("oz", 32, 56)])
def test_expired_wait_sets_the_error_and_recovers(prec, bit, mask):
    assert torch.cuda.is_available()
    import paper_2409_03904_b300 as mrhs
    lib = mrhs._lib.lib()
    L, nb, npts, R = (4, 4, 3, 3), 32, 81, 8
    disp, _ = stencil(npts)
    A = coarse_op(L, nb, npts, 9191, 14.0)
    X = vectors(L, nb, R, 9192)
    op = mrhs.CoarseOp(torch.from_numpy(A).cuda(), L, disp, (prec,))
    Xd = torch.from_numpy(X).cuda()
    if prec != "oz":
        Xd = Xd.to(torch.complex64)
    assert mrhs.device_error() == 0
    try:
        assert lib.mrhs_debug_wait_limit(1000) == 0            # 1 us
        for _ in range(2):
            op.apply(Xd, prec)
            err = mrhs.device_error()
            assert err & bit, err                              # the epilogue's wait ran out
            assert (err & ~mask) == 0, err                     # and only this kernel's roles
    finally:
        assert lib.mrhs_debug_wait_limit(0) == 0
    Y = op.apply(Xd, prec).cpu().numpy()
    assert mrhs.device_error() == 0
    if prec == "oz":
        assert rel(Y, coarse_op_apply(A, X, L, disp)) <= 1e-12
    else:
        assert rel(Y, lowprec_apply(A, X, L, disp, prec)) <= 1e-5
    assert lib.mrhs_debug_wait_limit(20_000_000_000) == -1     # above 10 s: rejected
