"""One rank's part of a decomposed lattice on the GPU (Sec. 2.6: input on the
padded local volume, output on the owned sites).

* mrhs_gather_rows / mrhs_scatter_rows against numpy indexing;
* the operator with an input halo (mrhs_op_create_halo) in FP64, DF32, FP32
  and OZ: for each rank of a 2- and a 4-rank grid, its padded input is
  filled straight from the global vector (no messages), and its output must
  equal the oracle's operator on the whole lattice at the owned sites;
* the decomposed BlockCGrQ driver (domain.block_cg with the library's
  kernels) on the one-rank grid with forced ghost layers, which exchange
  with themselves: equal to the oracle's BlockCGrQ on the whole lattice.
"""
import ctypes

import numpy as np
import pytest
import torch

from oracle.lowprec import quantise_op, quantise_vec
from oracle.ops import coarse_op_apply
from oracle.solvers import block_cg_rq
from synth import coarse_op, stencil, vectors

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


def test_gather_scatter_rows(mrhs):
    lib = mrhs._lib.lib()
    rng = np.random.default_rng(1)
    src = torch.from_numpy(rng.standard_normal((37, 5, 3)) + 1j * rng.standard_normal((37, 5, 3))).cuda()
    idx = np.array([4, 0, 36, 17, 17, 99, -1, 8], dtype=np.int64)     # two out of range
    di = torch.from_numpy(idx).cuda()
    rb = 5 * 3 * 16
    out = torch.full((8, 5, 3), 7.0 + 0j, dtype=torch.complex128, device="cuda")
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.mrhs_gather_rows(ctypes.c_void_p(src.data_ptr()), 37, ctypes.c_void_p(di.data_ptr()),
                                8, ctypes.c_void_p(out.data_ptr()), rb, s) == 0
    o = out.cpu().numpy()
    ok = (idx >= 0) & (idx < 37)
    assert np.array_equal(o[ok], src.cpu().numpy()[idx[ok]])
    assert np.all(o[~ok] == 7.0)                      # skipped rows untouched
    dst = torch.zeros((40, 5, 3), dtype=torch.complex128, device="cuda")
    sidx = np.array([3, 39, 0, 12, 50], dtype=np.int64)
    ds = torch.from_numpy(sidx).cuda()
    assert lib.mrhs_scatter_rows(ctypes.c_void_p(src.data_ptr()), 5, ctypes.c_void_p(ds.data_ptr()),
                                 ctypes.c_void_p(dst.data_ptr()), 40, rb, s) == 0
    d = dst.cpu().numpy()
    ref = np.zeros((40, 5, 3), dtype=np.complex128)
    ref[sidx[:4]] = src.cpu().numpy()[:4]
    assert np.array_equal(d, ref)
    assert lib.mrhs_gather_rows(ctypes.c_void_p(src.data_ptr()), 37, ctypes.c_void_p(di.data_ptr()),
                                8, ctypes.c_void_p(out.data_ptr()), 24, s) == -1   # not a multiple of 16


def padded_input(dom, X):
    """The padded input of a rank filled from the global vector: padded
    coordinate c -> global (c - h + q l) mod L."""
    Lin, h, q, l, L = (np.array(v) for v in (dom.Lin, dom.h, dom.q, dom.l, dom.L))
    i = np.arange(dom.Vin)
    c = np.stack([(i // np.prod(Lin[:mu])) % Lin[mu] for mu in range(4)], axis=-1)
    g = np.mod(c - h + q * l, L)
    gi = g[:, 0] + L[0] * (g[:, 1] + L[1] * (g[:, 2] + L[2] * g[:, 3]))
    return X[gi]


@pytest.mark.parametrize("grid", [(1, 1, 1, 2), (2, 1, 2, 1), (1, 2, 1, 1)])
@pytest.mark.parametrize("prec", ["fp64", "df32", "fp32", "oz"])
def test_halo_operator_on_each_rank(mrhs, grid, prec):
    from paper_2409_03904_b300 import domain
    L, nb, npts, R = (4, 4, 2, 4), 16, 81, 5
    disp, _ = stencil(npts)
    A = coarse_op(L, nb, npts, 5050, 20.0)
    X = vectors(L, nb, R, 5051)
    ref = coarse_op_apply(A, X, L, disp)
    if prec == "fp32":
        ref = coarse_op_apply(quantise_op(A, "fp32"), quantise_vec(X, "fp32"), L, disp)
    tol = {"fp64": 1e-13, "df32": 1e-11, "fp32": 1e-5, "oz": 1e-12}[prec]
    vdt = torch.complex64 if prec == "fp32" else torch.complex128
    for rank in range(int(np.prod(grid))):
        dom = domain.Domain(L, grid, rank)
        op = domain.halo_op(dom, torch.from_numpy(A[dom.global_sites]).cuda(), disp, (prec,))
        Xin = torch.from_numpy(padded_input(dom, X)).to(vdt).cuda()
        Y = op.apply(Xin, prec).cpu().numpy()
        assert Y.shape == (dom.V, nb, R)
        assert rel_per_rhs(Y, ref[dom.global_sites]) <= tol, (rank, prec)
    assert mrhs.device_error() == 0


def test_halo_operator_limits(mrhs):
    from paper_2409_03904_b300 import domain
    L, nb, npts = (4, 2, 2, 2), 8, 9
    disp, _ = stencil(npts)
    A = torch.from_numpy(coarse_op(L, nb, npts, 6060, 20.0)).cuda()
    dom = domain.Domain(L, (2, 1, 1, 1), 0)
    op = domain.halo_op(dom, A[torch.from_numpy(dom.global_sites).cuda()].contiguous(), disp,
                        ("fp64",))
    Xin = torch.zeros((dom.Vin, nb, 2), dtype=torch.complex128, device="cuda")
    with pytest.raises(mrhs.MrhsError):
        op.apply_dag(Xin, "fp64")                          # needs off-rank coefficients
    Xl = torch.zeros((dom.V, nb, 2), dtype=torch.complex128, device="cuda")
    with pytest.raises(mrhs.MrhsError):
        op.solve(Xl)                                        # whole-lattice entry point
    with pytest.raises(ValueError):
        op.apply(Xl, "fp64")                                # input must be padded
    with pytest.raises(mrhs.MrhsError):
        domain.halo_op(dom, A[torch.from_numpy(dom.global_sites).cuda()].contiguous(), disp,
                       ("fp16",))                           # tensor-core forms: whole lattice only


@pytest.mark.parametrize("prec", ["fp64", "oz"])
def test_decomposed_block_cg_one_rank(mrhs, prec):
    """The decomposed driver on the library's kernels: one rank, ghost layers
    forced in two dimensions (self exchange through the gather / scatter
    kernels), against the oracle's BlockCGrQ on the whole lattice."""
    from paper_2409_03904_b300 import domain
    L, nb, npts, R = (4, 3, 4, 3), 8, 81, 4
    disp, _ = stencil(npts)
    A = coarse_op(L, nb, npts, 7070, 30.0)
    B = vectors(L, nb, R, 7071)
    dom = domain.Domain(L, (1, 1, 1, 1), 0, pad=(0, 1, 0, 1))
    assert dom.h == (0, 1, 0, 1) and dom.Vin > dom.V
    op = domain.halo_op(dom, torch.from_numpy(A[dom.global_sites]).cuda(), disp, (prec,))
    be = domain.DeviceBackend(dom, op, prec)
    comm = domain.SelfComm()
    Bl = torch.from_numpy(B[dom.global_sites]).cuda()
    Y = domain.apply(dom, be, Bl, comm).cpu().numpy()
    assert rel_per_rhs(Y, coarse_op_apply(A, B, L, disp)[dom.global_sites]) <= 1e-12
    X, info = domain.block_cg(dom, be, comm, Bl, tol=1e-10, maxiter=500)
    Xo, io = block_cg_rq(lambda V: coarse_op_apply(A, V, L, disp), B, tol=1e-10, maxiter=500)
    assert info["converged"] and io["converged"]
    assert abs(info["iters"] - io["iters"]) <= 1
    assert rel_per_rhs(X.cpu().numpy(), Xo[dom.global_sites]) <= 1e-9
    r = B[dom.global_sites] - coarse_op_apply(A, X.cpu().numpy()[np.argsort(dom.global_sites)],
                                             L, disp)[dom.global_sites]
    bn = np.linalg.norm(B.reshape(-1, R), axis=0)
    assert np.max(np.linalg.norm(r.reshape(-1, R), axis=0) / bn) <= 1.5e-10
    assert mrhs.device_error() == 0
