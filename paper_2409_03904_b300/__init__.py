"""Multi-right-hand-side coarse-grid operator and block CG for NVIDIA B300.

Python face of libmrhs (include/mrhs.h); every computation runs in the CUDA
library, this package only marshals torch tensors.  Layouts: coefficients
A[x][p][a][b] complex128; vectors [V][nb][nrhs] (RHS fastest), complex128
for FP64 and complex64 for the FP32/BF16/FP16 operators.
"""
import ctypes
import os

import numpy as np
import torch

from . import _lib
from ._lib import (C64, C128, PREC, SOLVE_CG5D, SOLVE_FP64, SOLVE_MIXED, MrhsError, SolveInfo,
                   SolveParams)

__all__ = ["CoarseOp", "coarse_apply", "coarse_solve", "batch_apply", "batch_solve", "autotune",
           "autotune_save", "autotune_load", "autotune_entries", "autotune_clear", "block_inner",
           "block_project", "block_promote",
           "block_axpy", "herm_factor", "MrhsError", "PREC",
           "SOLVE_FP64", "SOLVE_MIXED", "block_tc", "device_error", "version"]


def launch_count():
    """Kernels launched by the library in this process so far."""
    return int(_lib.lib().mrhs_launch_count())


def version():
    return _lib.lib().mrhs_version().decode()


def block_tc(mode):
    """Complex64 block algebra of 4..32 columns on the tensor cores (1, the
    default) or on the FP32 FMA pipes (0); returns the previous mode."""
    r = int(_lib.lib().mrhs_block_tc(int(mode)))
    if r < 0:
        _lib.check(r)
    return r


def device_error():
    """Sticky error word of the tensor-core kernels (0 = none); clears it."""
    return int(_lib.lib().mrhs_device_error())


class CoarseOp:
    """Coarse operator H with Y(x) = sum_p A_p(x) X(x + delta_p).

    A: CUDA complex128 tensor [V][npts][nb][nb]; L: 4 lattice extents; disp:
    int8 [npts][4] displacements (disp[0] = 0); precisions: any of "fp64",
    "fp32", "bf16", "fp16", "fp16x", "tc32", "df32", "oz" ("df32" comes with
    "fp64" and implies it; "oz" is the digit-sliced tensor-core form of the
    FP64 operator and needs neither, except for its adjoint, which is built
    from the FP64 copy).  The operator keeps its own packed copies.
    """

    def __init__(self, A, L, disp, precisions=("fp64", "fp32"), halo=None):
        """halo: None, or 4 ints in {0, 1}: one rank's part of a decomposed
        lattice (mrhs_op_create_halo) -- L are the owned extents, inputs live
        on the padded lattice L + 2 halo, outputs on L; only apply() works."""
        l = _lib.lib()
        self.L = tuple(int(v) for v in L)
        self.V = int(np.prod(self.L))
        self.halo = tuple(int(v) for v in halo) if halo is not None else (0, 0, 0, 0)
        self.Lin = tuple(a + 2 * h for a, h in zip(self.L, self.halo))
        self.Vin = int(np.prod(self.Lin))
        disp = np.ascontiguousarray(np.asarray(disp, dtype=np.int8).reshape(-1, 4))
        self.npts = disp.shape[0]
        if A.dim() != 4 or A.shape[0] != self.V or A.shape[1] != self.npts or A.shape[2] != A.shape[3]:
            raise ValueError(f"A must be [V][npts][nb][nb], got {tuple(A.shape)}")
        self.nb = int(A.shape[2])
        self.N = self.V * self.nb
        precisions = tuple(precisions)
        if "fp64" in precisions and "df32" not in precisions:
            precisions += ("df32",)
        if "df32" in precisions and "fp64" not in precisions:
            precisions = ("fp64",) + precisions
        self.precisions = precisions
        mask = 0
        for p in self.precisions:
            mask |= 1 << PREC[p]
        Lc = (ctypes.c_int32 * 4)(*self.L)
        h = ctypes.c_void_p()
        with torch.cuda.device(A.device):
            if halo is None:
                _lib.check(l.mrhs_op_create(ctypes.byref(h), Lc, self.nb, self.npts,
                                            disp.ctypes.data_as(ctypes.c_void_p),
                                            _lib.dev_ptr(A, torch.complex128, "A"), mask,
                                            _lib.stream_ptr()))
            else:
                Hc = (ctypes.c_int32 * 4)(*self.halo)
                _lib.check(l.mrhs_op_create_halo(ctypes.byref(h), Lc, Hc, self.nb, self.npts,
                                                 disp.ctypes.data_as(ctypes.c_void_p),
                                                 _lib.dev_ptr(A, torch.complex128, "A"), mask,
                                                 _lib.stream_ptr()))
        self._h = h
        self.device = A.device
        self.disp = disp

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.lib().mrhs_op_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _apply(self, fn, X, prec, out):
        dt = _lib.vec_dtype(prec)
        if X.shape[:2] != (self.Vin, self.nb):
            raise ValueError(f"X must be [{self.Vin}][nb][nrhs], got {tuple(X.shape)}")
        if out is None:
            Y = torch.empty((self.V,) + tuple(X.shape[1:]), dtype=X.dtype, device=X.device)
        else:
            Y = out
            if Y.shape != (self.V,) + tuple(X.shape[1:]):
                raise ValueError("out must be [V][nb][nrhs]")
        fn(self._h, PREC[prec], _lib.dev_ptr(X, dt, "X"), _lib.dev_ptr(Y, dt, "Y"),
           int(X.shape[2]), _lib.stream_ptr())
        return Y

    def apply(self, X, prec="fp64", out=None):
        """Y = H X in precision `prec`."""
        l = _lib.lib()
        return self._apply(lambda *a: _lib.check(l.coarse_op_apply(*a)), X, prec, out)

    def apply_dag(self, X, prec="fp64", out=None):
        """Y = H^dagger X in precision `prec`."""
        l = _lib.lib()
        return self._apply(lambda *a: _lib.check(l.coarse_op_apply_dag(*a)), X, prec, out)

    def outer(self, G, X, alpha=1.0):
        """alpha * G(x) X(x + delta_p)^dagger on the stencil: complex128
        [V][npts][nb][nb] (the coefficient adjoint)."""
        if G.dtype != X.dtype or G.shape != X.shape:
            raise TypeError("G and X must have the same dtype and shape")
        GA = torch.empty((self.V, self.npts, self.nb, self.nb), dtype=torch.complex128,
                         device=G.device)
        _lib.check(_lib.lib().coarse_op_outer(self._h, _lib.dev_ptr(G, None, "G"),
                                              _lib.dev_ptr(X, None, "X"), _lib.dev_ptr(GA),
                                              float(alpha), int(G.shape[2]), _dtype_code(G),
                                              _lib.stream_ptr()))
        return GA

    def lambda_max(self, prec="fp32", iters=40):
        """Power-method estimate of the largest eigenvalue (cached on the op)."""
        lam = ctypes.c_double()
        _lib.check(_lib.lib().mrhs_op_lambda_max(self._h, PREC[prec], int(iters),
                                                 ctypes.byref(lam), _lib.stream_ptr()))
        return float(lam.value)

    def hermitian(self, mode=None):
        """Hermitian pairing of the tensor-core kernels (one coefficient tile
        per point pair, see mrhs_op_hermitian): None queries; 0 / False off,
        1 / True every tensor-core form, 2 TC32 only; off by default.
        Returns the mode after the call."""
        act = ctypes.c_int32()
        m = -1 if mode is None else int(mode)
        _lib.check(_lib.lib().mrhs_op_hermitian(self._h, m, ctypes.byref(act)))
        return int(act.value)

    def tc_tune(self, pts_per_stage=0, ctas_per_sm=1, max_stages=32):
        """Launch shape of the BF16/FP16 tensor-core kernel (0 = default)."""
        _lib.check(_lib.lib().mrhs_op_tc_tune(self._h, int(pts_per_stage), int(ctas_per_sm),
                                              int(max_stages)))

    def kernel_timing(self, enable=True):
        """Record CUDA events around every main operator kernel of this op."""
        _lib.check(_lib.lib().mrhs_op_kernel_timing(self._h, 1 if enable else 0))

    def kernel_time(self, prec):
        """(launches, summed ms) of the recorded main-kernel launches; clears."""
        n, ms = ctypes.c_int64(), ctypes.c_double()
        _lib.check(_lib.lib().mrhs_op_kernel_time(self._h, PREC[prec], ctypes.byref(n),
                                                  ctypes.byref(ms)))
        return int(n.value), float(ms.value)

    def cheby(self, X, lo, hi, order, prec="fp32", out=None):
        """P = p(H) X, p the Chebyshev interpolant of 1/x on [lo, hi]."""
        dt = _lib.vec_dtype(prec)
        P = torch.empty_like(X) if out is None else out
        _lib.check(_lib.lib().cheby_apply(self._h, PREC[prec], float(lo), float(hi), int(order),
                                          _lib.dev_ptr(X, dt, "X"), _lib.dev_ptr(P, dt, "P"),
                                          int(X.shape[2]), _lib.stream_ptr()))
        return P

    def coarsen(self, block, basis, disp):
        """Coarse operator of this (fine) operator on a blocked basis (Sec.
        3.4): A[b][p][j][k] = <phi_j^b | M | phi_k^(b + disp[p])> by the
        momentum-phase method.  block: 4 ints dividing L; basis: complex128
        [V_c][prod(block) nb][n_basis] (device); disp: [npts][4] in {-1,0,1}.
        Returns complex128 [V_c][npts][n_basis][n_basis] (device), ready for
        CoarseOp(A, L_c, disp)."""
        block = (ctypes.c_int32 * 4)(*[int(v) for v in block])
        disp = np.ascontiguousarray(np.asarray(disp, dtype=np.int8).reshape(-1, 4))
        Vc, vb, nbasis = (int(v) for v in basis.shape)
        bvol = int(np.prod(list(block)))
        if Vc * bvol != self.V or vb != bvol * self.nb:
            raise ValueError("basis must be [V / prod(block)][prod(block) * nb][n_basis]")
        A = torch.empty((Vc, disp.shape[0], nbasis, nbasis), dtype=torch.complex128,
                        device=basis.device)
        _lib.check(_lib.lib().coarsen_op(self._h, block, _lib.dev_ptr(basis, torch.complex128, "basis"),
                                         nbasis, disp.ctypes.data_as(ctypes.c_void_p), disp.shape[0],
                                         _lib.dev_ptr(A), _lib.stream_ptr()))
        return A

    def defl_cheby(self, U, lam, B, lo, hi, order, prec="fp64", out=None):
        """Deflated Chebyshev coarse solve (Sec. 2.3): U Lambda^-1 U^dagger B
        + p(H)(B - U U^dagger B), p the degree-`order` Chebyshev
        approximation of 1/x on [lo, hi].  U: [V][nb][n_ev] orthonormal
        eigenvectors (device), lam: their n_ev eigenvalues (host sequence),
        B: [V][nb][nrhs]; element type complex128 for fp64/df32, complex64
        otherwise."""
        dt = _lib.vec_dtype(prec)
        lam = np.ascontiguousarray(np.asarray(lam, dtype=np.float64).reshape(-1))
        n_ev = int(lam.size)
        if n_ev and (U.shape[:2] != (self.V, self.nb) or U.shape[2] != n_ev):
            raise ValueError("U must be [V][nb][n_ev]")
        X = torch.empty_like(B) if out is None else out
        uptr = _lib.dev_ptr(U, dt, "U") if n_ev else ctypes.c_void_p(None)
        _lib.check(_lib.lib().coarse_solve_defl_cheby(
            self._h, PREC[prec], uptr, lam.ctypes.data_as(ctypes.c_void_p), n_ev, float(lo),
            float(hi), int(order), _lib.dev_ptr(B, dt, "B"), _lib.dev_ptr(X, dt, "X"),
            int(B.shape[2]), _lib.stream_ptr()))
        return X

    def solve(self, B, X0=None, mode="fp64", raise_on_fail=True, **kw):
        """Block CG (Fig. 2) for H X = B; returns (X, info dict).

        mode "fp64": plain FP64 BlockCGrQ (precond=1 with precond_prec "fp64"
        for the FP64 Chebyshev-preconditioned form); mode "mixed": FP64-outer
        defect correction around a complex64 preconditioned block CG; mode
        "cg5d": one CG on the enlarged five-dimensional system (krylov_prec
        "fp64" or "df32").
        Keyword arguments override mrhs_solve_params fields.
        """
        l = _lib.lib()
        p = SolveParams()
        modes = {"fp64": SOLVE_FP64, "mixed": SOLVE_MIXED, "cg5d": SOLVE_CG5D}
        if mode not in modes:
            raise ValueError(f"mode must be one of {sorted(modes)}")
        l.mrhs_solve_params_default(ctypes.byref(p), modes[mode])
        for k, v in kw.items():
            if k in ("precond_prec", "krylov_prec", "residual_prec", "fp64_prec") and isinstance(v, str):
                v = PREC[v]
            if not hasattr(p, k):
                raise KeyError(k)
            setattr(p, k, v)
        X = torch.zeros_like(B) if X0 is None else X0.clone()
        info = SolveInfo()
        code = l.block_cg_solve(self._h, _lib.dev_ptr(B, torch.complex128, "B"),
                                _lib.dev_ptr(X, torch.complex128, "X"), int(B.shape[2]),
                                ctypes.byref(p), ctypes.byref(info), _lib.stream_ptr())
        if code not in (0, -3) or (code == -3 and raise_on_fail):
            _lib.check(code)
        return X, info.as_dict()


def _ptr_array(ts):
    return (ctypes.c_void_p * len(ts))(*[t.data_ptr() for t in ts])


def autotune(ops, prec, nrhs, reps=3):
    """Time launch shapes of the tensor-core kernel for `ops` (one operator,
    or a list solved as one batched launch) at `nrhs` right-hand sides (an
    int, or one per operator); cache and return the winner as a dict."""
    if isinstance(ops, CoarseOp):
        ops = [ops]
    if isinstance(nrhs, int):
        nrhs = [nrhs] * len(ops)
    l = _lib.lib()
    hs = (ctypes.c_void_p * len(ops))(*[o._h.value for o in ops])
    R = (ctypes.c_int32 * len(ops))(*[int(r) for r in nrhs])
    res = _lib.TuneResult()
    _lib.check(l.mrhs_autotune(hs, len(ops), PREC[prec], R, int(reps), ctypes.byref(res),
                               _lib.stream_ptr()))
    return res.as_dict()


def autotune_save(path):
    """Write the launch-shape cache to a text file."""
    _lib.check(_lib.lib().mrhs_autotune_save(os.fsencode(path)))


def autotune_load(path):
    """Merge a saved launch-shape cache into this process's cache."""
    _lib.check(_lib.lib().mrhs_autotune_load(os.fsencode(path)))


def autotune_entries():
    return int(_lib.lib().mrhs_autotune_entries())


def autotune_clear():
    _lib.lib().mrhs_autotune_clear()


def batch_apply(ops, Xs, prec="fp16"):
    """One persistent launch applying each ops[i] to Xs[i] (complex64)."""
    dt = _lib.vec_dtype(prec)
    Ys = [torch.empty_like(X) for X in Xs]
    for X in Xs:
        _lib.dev_ptr(X, dt, "X")
    hs = (ctypes.c_void_p * len(ops))(*[o._h.value for o in ops])
    R = (ctypes.c_int32 * len(ops))(*[int(X.shape[2]) for X in Xs])
    _lib.check(_lib.lib().mrhs_batch_apply(hs, len(ops), PREC[prec], _ptr_array(Xs),
                                           _ptr_array(Ys), R, _lib.stream_ptr()))
    return Ys


def batch_solve(ops, Bs, mode="mixed", raise_on_fail=True, **kw):
    """Solve ops[i] X_i = Bs[i] side by side; returns ([X_i], [info_i])."""
    l = _lib.lib()
    p = SolveParams()
    l.mrhs_solve_params_default(ctypes.byref(p), SOLVE_MIXED if mode == "mixed" else SOLVE_FP64)
    for k, v in kw.items():
        if k in ("precond_prec", "krylov_prec", "residual_prec", "fp64_prec") and isinstance(v, str):
            v = PREC[v]
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    for B in Bs:
        _lib.dev_ptr(B, torch.complex128, "B")
    Xs = [torch.zeros_like(B) for B in Bs]
    infos = (SolveInfo * len(ops))()
    hs = (ctypes.c_void_p * len(ops))(*[o._h.value for o in ops])
    R = (ctypes.c_int32 * len(ops))(*[int(B.shape[2]) for B in Bs])
    code = l.mrhs_batch_solve(hs, len(ops), _ptr_array(Bs), _ptr_array(Xs), R, ctypes.byref(p),
                              ctypes.cast(infos, ctypes.c_void_p), _lib.stream_ptr())
    if code not in (0, -3) or (code == -3 and raise_on_fail):
        _lib.check(code)
    return Xs, [i.as_dict() for i in infos]


def _dtype_code(t):
    if t.dtype == torch.complex128:
        return C128
    if t.dtype == torch.complex64:
        return C64
    raise TypeError("vectors must be complex128 or complex64")


def block_project(basis, F):
    """C[x] = basis[x]^dagger F[x] per coarse site x (Sec. 2.5.1): basis
    [n_blocks][v_block][n_basis], F [n_blocks][v_block][nrhs] -> C
    [n_blocks][n_basis][nrhs]; complex128 (FP64) or complex64 (FP32)."""
    nblk, vb, nbasis = (int(v) for v in basis.shape)
    if F.dtype != basis.dtype or F.shape[:2] != (nblk, vb):
        raise ValueError("F must be [n_blocks][v_block][nrhs] of the basis dtype")
    R = int(F.shape[2])
    C = torch.empty((nblk, nbasis, R), dtype=F.dtype, device=F.device)
    _lib.check(_lib.lib().block_project(_lib.dev_ptr(basis, None, "basis"), _lib.dev_ptr(F, None, "F"),
                                        _lib.dev_ptr(C), nblk, vb, nbasis, R, _dtype_code(F),
                                        _lib.stream_ptr()))
    return C


def block_promote(basis, C):
    """F[x] = basis[x] C[x] per coarse site x (Sec. 2.5.1): basis
    [n_blocks][v_block][n_basis], C [n_blocks][n_basis][nrhs] -> F
    [n_blocks][v_block][nrhs]; complex128 (FP64) or complex64 (FP32)."""
    nblk, vb, nbasis = (int(v) for v in basis.shape)
    if C.dtype != basis.dtype or C.shape[:2] != (nblk, nbasis):
        raise ValueError("C must be [n_blocks][n_basis][nrhs] of the basis dtype")
    R = int(C.shape[2])
    F = torch.empty((nblk, vb, R), dtype=C.dtype, device=C.device)
    _lib.check(_lib.lib().block_promote(_lib.dev_ptr(basis, None, "basis"), _lib.dev_ptr(C, None, "C"),
                                        _lib.dev_ptr(F), nblk, vb, nbasis, R, _dtype_code(C),
                                        _lib.stream_ptr()))
    return F


def block_inner(X, Y):
    """G = X^dagger Y (complex128 [rx][ry]) for [.., rx] and [.., ry] blocks."""
    if X.dtype != Y.dtype:
        raise TypeError("X and Y must share a dtype")
    rx, ry = int(X.shape[-1]), int(Y.shape[-1])
    N = X.numel() // rx
    if Y.numel() // ry != N:
        raise ValueError("row counts differ")
    G = torch.empty((rx, ry), dtype=torch.complex128, device=X.device)
    _lib.check(_lib.lib().block_inner(_lib.dev_ptr(X, None, "X"), _lib.dev_ptr(Y, None, "Y"),
                                      _lib.dev_ptr(G), N, rx, ry, _dtype_code(X),
                                      _lib.stream_ptr()))
    return G


def block_axpy(Y, X, M, beta=0.0):
    """Y <- beta Y + X M in place (M complex128 [rin][rout] on the device)."""
    rin, rout = int(X.shape[-1]), int(Y.shape[-1])
    N = X.numel() // rin
    if X.dtype != Y.dtype:
        raise TypeError("X and Y must share a dtype")
    M = M.to(device=X.device, dtype=torch.complex128).contiguous()
    _lib.check(_lib.lib().block_axpy(_lib.dev_ptr(Y, None, "Y"), _lib.dev_ptr(X, None, "X"),
                                     _lib.dev_ptr(M), float(beta), N, rin, rout, _dtype_code(X),
                                     _lib.stream_ptr()))
    return Y


def herm_factor(G, tau=1e-12):
    """(S, W, rank) with T = Q S and T W = Q for the Gram G = T^dagger T."""
    r = int(G.shape[0])
    G = G.to(torch.complex128).contiguous()
    S = torch.empty_like(G)
    W = torch.empty_like(G)
    rank = torch.zeros(1, dtype=torch.int32, device=G.device)
    _lib.check(_lib.lib().herm_factor(_lib.dev_ptr(G), _lib.dev_ptr(S), _lib.dev_ptr(W),
                                      _lib.dev_ptr(rank), r, float(tau), _lib.stream_ptr()))
    return S, W, int(rank.item())


from .autograd import coarse_apply, coarse_solve  # noqa: E402
