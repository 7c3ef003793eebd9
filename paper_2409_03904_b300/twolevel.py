"""Two-level (ADEF2) multigrid preconditioning and the two outer solvers the
paper compares: flexible ADEF2 CG (Fig. 1) with the original, variable
preconditioner, against Preconditioned BlockCGrQ (Fig. 2 right) with the
stationary one of Sec. 2.3.

Fig. 1 and Sec. 2:
* coarse-grid correction Q = P h^-1 P^dagger: project the fine vector onto
  the blocked basis (block_project), solve with the coarse operator h,
  promote back (block_promote);
* preconditioner M^-1 = P_R S + Q = S + Q (1 - H S), P_R = 1 - Q H, with a
  smoother S;
* the flexible CG of Fig. 1 on every right-hand side (run here as
  independent processes advancing in lockstep, each column with its own
  scalars: mrhs_col_dot / mrhs_col_ratio / mrhs_col_update).

The two preconditioners (Sec. 2 and Sec. 2.3):
* variable (``krylov``): S = a fixed number of CG iterations on the
  infra-red shifted operator H + Lambda (7 and 2.0 in the paper), one CG
  process per right-hand side; h^-1 = CG from the deflated start
  U Lambda_ev^-1 U^dagger c to a loose residual (4e-2 in the paper);
* stationary (``stationary``): S = the Chebyshev approximation to 1/x of
  order 8 on [lo, hi] (cheby_apply), h^-1 = the deflated Chebyshev solve
  Q^{Cheby+defl} (coarse_solve_defl_cheby).

Readings of Fig. 1: y_k in step 9 is z_k; the
orthogonalisation of step 8 is flexible CG's H-projection of the new
direction onto the last m_max directions, c_i = (p_i, H p_k)/(p_i, H p_i),
applied to p_k and to its image w_k = H p_k.

Every step runs in the library's kernels; the host only keeps the loop,
reads the residual norms (one small read per iteration) and decides which
columns have converged.  Fine vectors use the coarse-vector layout
[V][nb][nrhs] of the fine lattice; the blocked layout that block_project
and block_promote take ([n_blocks][v_block][nrhs], the sites of a block
first-direction fastest) is reached with mrhs_gather_rows /
mrhs_scatter_rows.
"""
import numpy as np
import torch

from . import _lib


def _lib_():
    return _lib.lib()


def _code(t):
    return _lib.C128 if t.dtype == torch.complex128 else _lib.C64


def col_dot(X, Y):
    """out[j] = X[:, j]^dagger Y[:, j] (device complex128 [R])."""
    R = int(X.shape[-1])
    out = torch.empty(R, dtype=torch.complex128, device=X.device)
    _lib.check(_lib_().mrhs_col_dot(_lib.dev_ptr(X), _lib.dev_ptr(Y), _lib.dev_ptr(out),
                                    X.numel() // R, R, _code(X), _lib.stream_ptr()))
    return out


def col_ratio(num, den, scale=1.0, active=None):
    """scale * num / den per column (0 where den is 0 or the column is inactive)."""
    out = torch.empty_like(num)
    act = _lib.dev_ptr(active) if active is not None else ctypes_null()
    _lib.check(_lib_().mrhs_col_ratio(_lib.dev_ptr(num), _lib.dev_ptr(den), _lib.dev_ptr(out),
                                      act, int(num.numel()), float(scale), _lib.stream_ptr()))
    return out


def col_update(Y, X, coef, beta):
    """Y[:, j] = beta Y[:, j] + coef[j] X[:, j] in place."""
    R = int(Y.shape[-1])
    _lib.check(_lib_().mrhs_col_update(_lib.dev_ptr(Y), _lib.dev_ptr(X), _lib.dev_ptr(coef),
                                       float(beta), Y.numel() // R, R, _code(Y),
                                       _lib.stream_ptr()))
    return Y


def ctypes_null():
    import ctypes
    return ctypes.c_void_p(None)


def _const(R, v, dev):
    return torch.full((R,), complex(v), dtype=torch.complex128, device=dev)


def _norms(X):
    """Column norms, read back to the host."""
    return np.sqrt(np.maximum(col_dot(X, X).real.cpu().numpy(), 0.0))


def cg_columns(apply_H, B, X0=None, iters=None, tol=None, maxiter=1000, stats=None):
    """Plain CG on every column of B as an independent process, all columns
    in lockstep.  ``iters``: a fixed number of iterations (the smoother; an
    exhausted column, zero residual, stays put); ``tol``: each column stops
    once its recurrence residual |r_j| <= tol |b_j| (checked before each
    iteration), at most ``maxiter``
    iterations (a zero column stays zero).  Returns X; ``stats`` (a dict,
    optional) receives the number of iterations run."""
    R, dev = int(B.shape[-1]), B.device
    ones, mones = _const(R, 1.0, dev), _const(R, -1.0, dev)
    if X0 is None:
        X = torch.zeros_like(B)
        r = B.clone()
    else:
        X = X0.clone()
        r = B.clone()
        col_update(r, apply_H(X), mones, 1.0)
    p = r.clone()
    rr = col_dot(r, r)
    active = None
    bn = _norms(B) if tol is not None else None
    n = iters if iters is not None else maxiter
    k = 0
    for k in range(n + 1):
        if k == n:
            break
        if tol is not None:
            live = np.sqrt(np.maximum(rr.real.cpu().numpy(), 0.0)) > tol * bn
            if not live.any():
                break
            active = torch.from_numpy(live.astype(np.int32)).to(dev)
        w = apply_H(p)
        pw = col_dot(p, w)
        col_update(X, p, col_ratio(rr, pw, 1.0, active), 1.0)
        col_update(r, w, col_ratio(rr, pw, -1.0, active), 1.0)
        rr_new = col_dot(r, r)
        col_update(p, p, col_ratio(rr_new, rr, 1.0, active), 0.0)      # beta p
        col_update(p, r, ones, 1.0)                                      # + r
        rr = rr_new
    if stats is not None:
        stats["iters"] = k
    return X


class Transfer:
    """Project / promote between a fine lattice vector [V][nb][R] and the
    coarse one [V_c][n_basis][R] through the blocked basis
    [V_c][v_block][n_basis] (v_block = prod(block) * nb, rows i * nb + a for
    the site at position i of the block, first direction fastest): the same
    layout coarsen_op takes."""

    def __init__(self, L, block, nb, basis):
        self.L, self.block, self.nb = tuple(L), tuple(block), nb
        self.basis = basis
        Lc = tuple(l // b for l, b in zip(L, block))
        Vc, bv = int(np.prod(Lc)), int(np.prod(block))
        # coordinates of the coarse sites and of the positions inside a block
        # (first direction fastest); fine site of (coarse site, position)
        cc = np.stack([(np.arange(Vc) // int(np.prod(Lc[:m]))) % Lc[m] for m in range(4)], -1)
        ib = np.stack([(np.arange(bv) // int(np.prod(block[:m]))) % block[m] for m in range(4)], -1)
        g = cc[:, None, :] * np.asarray(block) + ib[None, :, :]              # [Vc][bv][4]
        site = g[..., 0] + L[0] * (g[..., 1] + L[1] * (g[..., 2] + L[2] * g[..., 3]))
        self.order = torch.from_numpy(site.reshape(-1).astype(np.int64)).to(basis.device)
        self.Vc, self.bv, self.V = Vc, bv, int(np.prod(L))

    def project(self, F):
        R = int(F.shape[-1])
        blk = torch.empty((self.Vc * self.bv, self.nb, R), dtype=F.dtype, device=F.device)
        _lib.check(_lib_().mrhs_gather_rows(_lib.dev_ptr(F), self.V, _lib.dev_ptr(self.order),
                                            self.Vc * self.bv, _lib.dev_ptr(blk),
                                            self.nb * R * F.element_size(), _lib.stream_ptr()))
        from . import block_project
        return block_project(self.basis, blk.view(self.Vc, self.bv * self.nb, R))

    def promote(self, C):
        R = int(C.shape[-1])
        from . import block_promote
        blk = block_promote(self.basis, C)
        F = torch.empty((self.V, self.nb, R), dtype=C.dtype, device=C.device)
        _lib.check(_lib_().mrhs_scatter_rows(_lib.dev_ptr(blk), self.Vc * self.bv,
                                             _lib.dev_ptr(self.order), _lib.dev_ptr(F), self.V,
                                             self.nb * R * C.element_size(), _lib.stream_ptr()))
        return F


class TwoLevel:
    """ADEF2 preconditioners on a fine operator ``fine`` (CoarseOp of the
    fine lattice, FP64 built), a Transfer and the coarse operator
    ``coarse`` (CoarseOp on the coarse lattice, e.g. from fine.coarsen),
    both applied in precision ``prec`` ("fp64")."""

    def __init__(self, fine, transfer, coarse, prec="fp64"):
        self.fine, self.T, self.coarse, self.prec = fine, transfer, coarse, prec

    def H(self, X):
        return self.fine.apply(X, self.prec)

    def Q(self, r, coarse_solve):
        return self.T.promote(coarse_solve(self.T.project(r)))

    def adef2(self, smoother, coarse_solve):
        """M^-1 r = t + Q (r - H t), t = S r (Fig. 1, step 2)."""
        def apply(r):
            t = smoother(r)
            v = r.clone()
            col_update(v, self.H(t), _const(r.shape[-1], -1.0, r.device), 1.0)
            col_update(t, self.Q(v, coarse_solve), _const(r.shape[-1], 1.0, r.device), 1.0)
            return t
        return apply

    # ---- the stationary preconditioner (Sec. 2.3)
    def chebyshev_smoother(self, lo, hi, order=8):
        return lambda r: self.fine.cheby(r, lo, hi, order, self.prec)

    def defl_cheby_solve(self, U, lam, lo, hi, order):
        return lambda c: self.coarse.defl_cheby(U, lam, c, lo, hi, order, self.prec)

    def stationary(self, smooth=(2.0, None, 8), defl=None):
        """smooth = (lo, hi, order) of the Chebyshev smoother; defl = (U,
        lam, lo, hi, order) of the deflated Chebyshev coarse solve."""
        return self.adef2(self.chebyshev_smoother(*smooth), self.defl_cheby_solve(*defl))

    # ---- the variable preconditioner (Sec. 2, the original HDCG)
    def shifted_cg_smoother(self, shifted, iters=7):
        """``iters`` CG iterations per column on ``shifted`` (a CoarseOp of
        H + Lambda)."""
        return lambda r: cg_columns(lambda v: shifted.apply(v, self.prec), r, iters=iters)

    def deflated_cg_solve(self, U, lam, tol=4e-2, maxiter=500):
        """CG per column on the coarse operator from the deflated start
        U Lambda^-1 U^dagger c (U: [V_c][n_b][n_ev], n_ev <= 64)."""
        from . import block_axpy, block_inner
        n_ev = int(U.shape[-1])
        if n_ev > 64:
            raise ValueError("deflated CG start: at most 64 eigenvectors")
        Ul = U.clone()
        inv = torch.as_tensor(1.0 / np.asarray(lam, dtype=np.float64),
                              dtype=torch.complex128).to(U.device)
        col_update(Ul, U, inv, 0.0)                                     # U Lambda^-1

        def solve(c):
            G = block_inner(U, c)                                       # U^dagger c
            X0 = block_axpy(torch.empty_like(c), Ul, G, 0.0)
            return cg_columns(lambda v: self.coarse.apply(v, self.prec), c, X0=X0, tol=tol,
                              maxiter=maxiter)
        return solve

    def krylov(self, shifted, iters=7, U=None, lam=None, tol=4e-2, maxiter=500):
        return self.adef2(self.shifted_cg_smoother(shifted, iters),
                          self.deflated_cg_solve(U, lam, tol, maxiter))


def flex_adef2(apply_H, apply_Minv, coarse, B, tol=1e-8, maxiter=1000, mmax=1):
    """Flexible ADEF2 CG (Fig. 1) on every column of B, the columns
    advancing in lockstep with their own scalars; a converged column is
    frozen (its step lengths become zero).  ``coarse`` applies Q for the
    start x_0 = Q b.  Returns (X, info) with per-column iteration counts
    and true relative residuals."""
    R, dev = int(B.shape[-1]), B.device
    ones = _const(R, 1.0, dev)
    mones = _const(R, -1.0, dev)
    bn = _norms(B)
    if not np.all(bn > 0):
        raise ValueError("flex_adef2: every right-hand side must be nonzero")
    X = coarse(B)                                                      # x_0 = Q b
    r = B.clone()
    col_update(r, apply_H(X), mones, 1.0)
    rn = _norms(r)
    iters = np.zeros(R, dtype=np.int64)
    live = rn > tol * bn
    active = torch.from_numpy(live.astype(np.int32)).to(dev)
    z = apply_Minv(r)
    p = z.clone()
    rz = col_dot(r, z)
    hist = []
    k = 0
    for k in range(1, maxiter + 1):
        if not live.any():
            k -= 1
            break
        d = apply_H(p)
        w = d.clone()
        for pi, wi in (hist[-mmax:] if mmax > 0 else []):
            nc = col_ratio(col_dot(pi, d), col_dot(pi, wi), -1.0)
            col_update(p, pi, nc, 1.0)
            col_update(w, wi, nc, 1.0)
        pw = col_dot(p, w)
        col_update(X, p, col_ratio(rz, pw, 1.0, active), 1.0)
        col_update(r, w, col_ratio(rz, pw, -1.0, active), 1.0)
        if mmax > 0:
            hist.append((p.clone(), w.clone()))
            hist = hist[-mmax:]
        iters[live] = k
        rn = _norms(r)
        live = live & (rn > tol * bn)
        if not live.any():
            break
        active = torch.from_numpy(live.astype(np.int32)).to(dev)
        z = apply_Minv(r)
        rz_new = col_dot(r, z)
        col_update(p, p, col_ratio(rz_new, rz, 1.0, active), 0.0)      # beta p
        col_update(p, z, ones, 1.0)                                      # + z
        rz = rz_new
    rt = B.clone()
    col_update(rt, apply_H(X), mones, 1.0)
    res = _norms(rt) / bn
    return X, dict(iters=int(iters.max()) if R else 0, col_iters=[int(v) for v in iters],
                   resid=[float(v) for v in res],
                   converged=bool(np.all(res <= 10 * tol) and not live.any()))


def prec_block_cg(apply_H, apply_Minv, B, tol=1e-8, maxiter=1000, tau=1e-14):
    """Preconditioned BlockCGrQ (Fig. 2 right) with a general preconditioner,
    on the library's block kernels (the library's own block_cg_solve takes
    the Chebyshev preconditioner only).  Readings as the library's: X update
    carries C_k, one factor S^dagger S = T^dagger t per iteration, Grams
    symmetrised before factorising; stop when |q C e_r| <= tol |b_r| for
    every column, then report true residuals.  Returns (X, info)."""
    from . import block_axpy, block_inner, herm_factor
    R, dev = int(B.shape[-1]), B.device
    eye = torch.eye(R, dtype=torch.complex128, device=dev)

    def mm(A, Bm):
        out = torch.empty((A.shape[0], Bm.shape[1]), dtype=torch.complex128, device=dev)
        return block_axpy(out, A.contiguous(), Bm, 0.0)

    def adj(A):
        return block_inner(A.contiguous(), eye)

    def factor(G):
        S, W, rank = herm_factor(G, tau)
        if rank < R:
            raise _lib.MrhsError(-4, f"prec_block_cg: the block lost rank ({rank} of {R})")
        return S, W

    bn = _norms(B)
    if not np.all(bn > 0):
        raise ValueError("prec_block_cg: every right-hand side must be nonzero")
    X = torch.zeros_like(B)
    r0 = B.clone()                                                      # z_0 = B - H X_0
    Z0 = apply_Minv(r0)
    C, Ci = factor(block_inner(Z0, r0))                                 # C^dag C = Z_0^dag r_0
    q = block_axpy(torch.empty_like(B), r0, Ci, 0.0)
    Q = block_axpy(torch.empty_like(B), Z0, Ci, 0.0)
    D = Q.clone()
    t = torch.empty_like(B)
    T = torch.empty_like(B)
    k, converged = 0, False
    for k in range(1, maxiter + 1):
        z = apply_H(D)                                                  # z_k = H D_k
        Zz = apply_Minv(z)                                              # Z_k = M^-1 z_k
        _, W1 = factor(block_inner(D, z))
        Nk = mm(W1, adj(W1))                                            # [D^dag z]^-1
        block_axpy(X, D, mm(Nk, C), 1.0)                                # X + D N C
        mN = mm(Nk, -eye)
        t.copy_(q)
        block_axpy(t, z, mN, 1.0)                                       # t = q - z N
        T.copy_(Q)
        block_axpy(T, Zz, mN, 1.0)                                      # T = Q - Z N
        S, Si = factor(block_inner(T, t))                               # S^dag S = T^dag t
        block_axpy(q, t, Si, 0.0)
        block_axpy(Q, T, Si, 0.0)
        block_axpy(T, D, adj(S), 0.0)                                   # D S^dag
        D.copy_(Q)
        block_axpy(D, T, eye, 1.0)                                      # D = Q + D S^dag
        C = mm(S, C)
        # |q C e_r|^2 = (C^dag (q^dag q) C)_rr
        E = mm(adj(C), mm(block_inner(q, q), C))
        est = np.sqrt(np.maximum(E.diagonal().real.cpu().numpy(), 0.0)) / bn
        if np.all(est <= tol):
            converged = True
            break
    rt = B.clone()
    block_axpy(rt, apply_H(X), -eye, 1.0)
    res = _norms(rt) / bn
    return X, dict(iters=k, resid=[float(v) for v in res],
                   converged=bool(converged and np.all(res <= 10 * tol)))
