"""torch.autograd wrappers of the coarse operator and of block_cg_solve.

The backward passes call the library's adjoint kernels (argument marshalling
and autograd bookkeeping only here):
* coarse_apply:  grad X = H^dagger grad Y (coarse_op_apply_dag),
                 grad A = grad Y X^dagger on the stencil (coarse_op_outer);
* coarse_solve:  grad B = H^-1 grad X (block CG again: H is Hermitian, so
                 H^-dagger = H^-1), grad A = -grad B X^dagger on the stencil.
                 B may be complex128 or complex64; a complex64 B gives a
                 complex64 X and grad B (the solve itself runs on complex128
                 vectors, in the mode the options choose, e.g. "mixed").
Coefficients A are complex128 [V][npts][nb][nb]; each entry is an independent
parameter (a perturbation that breaks Hermiticity is outside what the solve
accepts, so finite-difference checks of the solve use Hermitian directions).
"""
import torch

from . import CoarseOp


class _Apply(torch.autograd.Function):
    @staticmethod
    def forward(ctx, A, X, L, disp, prec):
        precs = ("fp64",) if prec == "fp64" else ("fp64", prec)
        op = CoarseOp(A.detach().contiguous(), L, disp, precs)
        Y = op.apply(X.detach().contiguous(), prec)
        ctx.op, ctx.prec = op, prec
        ctx.save_for_backward(X)
        return Y

    @staticmethod
    def backward(ctx, gY):
        (X,) = ctx.saved_tensors
        gY = gY.contiguous()
        gA = gX = None
        if ctx.needs_input_grad[1]:
            gX = ctx.op.apply_dag(gY, ctx.prec)
        if ctx.needs_input_grad[0]:
            gA = ctx.op.outer(gY, X.detach().contiguous(), 1.0)
        return gA, gX, None, None, None


class _Solve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, A, B, L, disp, opts):
        op = CoarseOp(A.detach().contiguous(), L, disp, opts.pop("precisions", ("fp64", "fp32")))
        X, info = op.solve(B.detach().to(torch.complex128).contiguous(), **opts)
        ctx.op, ctx.opts, ctx.dtype = op, opts, B.dtype
        ctx.save_for_backward(X)
        ctx.info = info
        return X.to(B.dtype)

    @staticmethod
    def backward(ctx, gX):
        (X,) = ctx.saved_tensors
        gB, _ = ctx.op.solve(gX.to(torch.complex128).contiguous(), **ctx.opts)
        gA = ctx.op.outer(gB, X, -1.0) if ctx.needs_input_grad[0] else None
        return gA, (gB.to(ctx.dtype) if ctx.needs_input_grad[1] else None), None, None, None


def coarse_apply(A, X, L, disp, prec="fp64"):
    """Y = H X with autograd through A and X (prec: fp64, fp32, bf16, fp16, ...)."""
    return _Apply.apply(A, X, tuple(L), disp, prec)


def coarse_solve(A, B, L, disp, **opts):
    """X = H^-1 B by block_cg_solve with autograd through A and B; keyword
    arguments go to CoarseOp.solve (plus `precisions` for the operator)."""
    return _Solve.apply(A, B, tuple(L), disp, dict(opts))
