"""Block CG family, Chebyshev preconditioner and spectral estimates, complex128.

Test infrastructure only (see the package docstring).

``apply_H`` and ``apply_Minv`` are callables on [V][nb][k] (or [N][k]) arrays.
Column r of B is right-hand side r; per-RHS stopping is relative to ||b_r||.

Readings of Fig. 2 taken here (the paper prints these steps tersely):
* X update carries C_k: X_{k+1} = X_k + D_k M_k C_k (left) and
  X_{k+1} = X_k + D_k N_k C_k (right).  With R_k = Q_k C_k this is what makes
  B - H X_{k+1} = Q_{k+1} C_{k+1}; without C_k the printed update solves for
  Q_0 instead of B.
* Right figure, step 12: one factor per iteration, S_k^dagger S_k = T_k^dagger t_k,
  used in steps 13-15 (the printed S_{k+1} on the left of step 12 is taken
  as S_k).
* z_0 (the residual) and z_k = H D_k are kept apart as r0 and z.
* The Gram entering a Cholesky is Hermitian-symmetrised first.
* Rank loss of the block (dependent right-hand sides, or the block Krylov
  space running out near finite termination) is handled by dropping the
  numerically null directions (``chol.block_factor``); the block then
  narrows and C becomes rectangular (k x nrhs).
* Stop when every active column satisfies ||b_r - H x_r|| <= tol ||b_r||;
  the loop uses the recurrence estimate ||(q C) e_r|| and the exit is
  confirmed on the true residual.
* A zero column b_r gives x_r = 0 and is removed from the block.
"""
import numpy as np

from .chol import block_factor, hpd_inverse
from .ops import as_matrix, column_norms


def _restore(X, shape):
    return X.reshape(shape)


def block_cg_rq(apply_H, B, X0=None, tol=1e-10, maxiter=1000, history=None):
    """BlockCGrQ (Fig. 2 left; Dubrulle 2001, Birk 2015) on H X = B.

    Returns (X, info) with info = {iters, converged, resid (true, relative)}.
    If ``history`` is a list, per-iteration dicts (X, Q, C, D, Z) are appended.
    """
    shape = B.shape
    Bm = as_matrix(B).astype(np.complex128)
    X = np.zeros_like(Bm) if X0 is None else as_matrix(X0).astype(np.complex128).copy()
    bn = column_norms(Bm)
    active = np.nonzero(bn > 0)[0]
    X[:, bn == 0] = 0.0
    info = dict(iters=0, converged=True, resid=np.zeros(Bm.shape[1]))
    if active.size == 0:
        return _restore(X, shape), info
    H = lambda V: as_matrix(apply_H(V.reshape(shape[:-1] + (V.shape[1],))))  # noqa: E731
    Xa = X[:, active]
    Ba = Bm[:, active]
    R0 = Ba - H(Xa)
    C, W = block_factor(np.conj(R0.T) @ R0)                      # R0 = Q0 C0
    Q = R0 @ W
    D = Q.copy()
    k = 0
    converged = False
    for k in range(1, maxiter + 1):
        Z = H(D)                                                 # Z_k = H D_k
        M = hpd_inverse(np.conj(D.T) @ Z)                        # M_k = [D^dag Z]^-1
        Xa = Xa + D @ (M @ C)                                    # X + D M C
        T = Q - Z @ M                                            # Q_k - Z_k M_k
        S, W = block_factor(np.conj(T.T) @ T)                    # = Q_{k+1} S_{k+1}
        Q = T @ W
        D = Q + D @ np.conj(S.T)                                 # D_{k+1}
        C = S @ C                                                # C_{k+1}
        if history is not None:
            history.append(dict(X=Xa.copy(), Q=Q.copy(), C=C.copy(), D=D.copy(), Z=Z.copy()))
        est = column_norms(C) / bn[active]
        if np.all(est <= tol) or C.shape[0] == 0:
            converged = True
            break
    X[:, active] = Xa
    true = column_norms(Bm - H(X))
    info["iters"] = k
    info["resid"] = np.where(bn > 0, true / np.where(bn > 0, bn, 1.0), 0.0)
    info["converged"] = bool(converged and np.all(info["resid"][active] <= 10 * tol))
    return _restore(X, shape), info


def prec_block_cg_rq(apply_H, apply_Minv, B, X0=None, tol=1e-10, maxiter=1000, history=None):
    """Preconditioned BlockCGrQ (Fig. 2 right): BlockCGrQ for M^-1 H in the
    M inner product, with the Cholesky kept explicit and both the
    unpreconditioned (q, z) and preconditioned (Q, Z) blocks rotated."""
    shape = B.shape
    Bm = as_matrix(B).astype(np.complex128)
    X = np.zeros_like(Bm) if X0 is None else as_matrix(X0).astype(np.complex128).copy()
    bn = column_norms(Bm)
    active = np.nonzero(bn > 0)[0]
    X[:, bn == 0] = 0.0
    info = dict(iters=0, converged=True, resid=np.zeros(Bm.shape[1]))
    if active.size == 0:
        return _restore(X, shape), info

    def H(V):
        return as_matrix(apply_H(V.reshape(shape[:-1] + (V.shape[1],))))

    def Minv(V):
        return as_matrix(apply_Minv(V.reshape(shape[:-1] + (V.shape[1],))))

    Xa = X[:, active]
    Ba = Bm[:, active]
    r0 = Ba - H(Xa)                                              # z_0 = B - H X_0
    Z0 = Minv(r0)                                                # Z_0 = M^-1 z_0
    C, Ci = block_factor(np.conj(Z0.T) @ r0)                     # C^dag C = Z_0^dag z_0
    q = r0 @ Ci
    Q = Z0 @ Ci
    D = Q.copy()
    k = 0
    converged = False
    for k in range(1, maxiter + 1):
        z = H(D)                                                 # z_k = H D_k
        Zz = Minv(z)                                             # Z_k = M^-1 z_k
        N = hpd_inverse(np.conj(D.T) @ z)                        # N_k = [D^dag z]^-1
        Xa = Xa + D @ (N @ C)                                    # X + D N C
        t = q - z @ N
        T = Q - Zz @ N
        S, Si = block_factor(np.conj(T.T) @ t)                   # S^dag S = T^dag t
        q = t @ Si
        Q = T @ Si
        D = Q + D @ np.conj(S.T)
        C = S @ C
        if history is not None:
            history.append(dict(X=Xa.copy(), q=q.copy(), Q=Q.copy(), C=C.copy(), D=D.copy()))
        est = column_norms(q @ C) / bn[active]                   # residual = q_k C_k
        if np.all(est <= tol) or C.shape[0] == 0:
            converged = True
            break
    X[:, active] = Xa
    true = column_norms(Bm - H(X))
    info["iters"] = k
    info["resid"] = np.where(bn > 0, true / np.where(bn > 0, bn, 1.0), 0.0)
    info["converged"] = bool(converged and np.all(info["resid"][active] <= 10 * tol))
    return _restore(X, shape), info


def cg(apply_H, b, x0=None, tol=1e-10, maxiter=1000, history=None):
    """Plain conjugate gradients (Hestenes-Stiefel) for one right-hand side."""
    b = np.asarray(b, dtype=np.complex128).reshape(-1)
    x = np.zeros_like(b) if x0 is None else np.asarray(x0, dtype=np.complex128).reshape(-1).copy()
    r = b - apply_H(x)
    p = r.copy()
    rr = np.vdot(r, r).real
    bn = np.linalg.norm(b)
    k = 0
    for k in range(1, maxiter + 1):
        Ap = apply_H(p)
        alpha = rr / np.vdot(p, Ap).real
        x = x + alpha * p
        r = r - alpha * Ap
        rr_new = np.vdot(r, r).real
        if history is not None:
            history.append(dict(x=x.copy(), r=r.copy()))
        if np.sqrt(rr_new) <= tol * bn:
            break
        p = r + (rr_new / rr) * p
        rr = rr_new
    return x, dict(iters=k, resid=np.linalg.norm(b - apply_H(x)) / bn)


def cheby_coeffs(lo, hi, order):
    """Chebyshev interpolant of f(x) = 1/x on [lo, hi] (Sec. 2.3): with
    m' = order + 1 nodes y_k = cos(pi (k + 1/2)/m'), x_k = ((hi-lo) y_k + hi + lo)/2,
    c_j = (2/m') sum_k f(x_k) T_j(y_k), and c_0 halved."""
    m1 = order + 1
    k = np.arange(m1)
    y = np.cos(np.pi * (k + 0.5) / m1)
    x = 0.5 * ((hi - lo) * y + hi + lo)
    f = 1.0 / x
    c = np.array([(2.0 / m1) * np.sum(f * np.cos(j * np.pi * (k + 0.5) / m1)) for j in range(m1)])
    c[0] *= 0.5
    return c


def cheby_eval_scalar(lam, lo, hi, order):
    """p(lambda) for scalars, summing c_j T_j(t) with T_j(t) = cos(j arccos t)
    inside [-1, 1] and cosh(j arccosh |t|) (with sign) outside."""
    c = cheby_coeffs(lo, hi, order)
    t = (2.0 * np.asarray(lam, dtype=np.float64) - (hi + lo)) / (hi - lo)
    out = np.zeros_like(t)
    for j, cj in enumerate(c):
        out = out + cj * _cheb_T(j, t)
    return out


def _cheb_T(j, t):
    t = np.asarray(t, dtype=np.float64)
    inside = np.abs(t) <= 1.0
    res = np.empty_like(t)
    res[inside] = np.cos(j * np.arccos(t[inside]))
    o = ~inside
    res[o] = np.sign(t[o]) ** j * np.cosh(j * np.arccosh(np.abs(t[o])))
    return res


def cheby_apply(apply_H, V, lo, hi, order):
    """p(H) V = sum_j c_j T_j(t(H)) V with t(H) = (2H - (hi+lo))/(hi-lo),
    by the three-term recurrence T_{j+1} = 2 t T_j - T_{j-1} (Sec. 2.3)."""
    c = cheby_coeffs(lo, hi, order)
    a = 2.0 / (hi - lo)
    b = -(hi + lo) / (hi - lo)
    Tm = V.astype(np.complex128)
    acc = c[0] * Tm
    if order == 0:
        return acc
    T = a * apply_H(Tm) + b * Tm
    acc = acc + c[1] * T
    for j in range(2, order + 1):
        Tn = 2.0 * (a * apply_H(T) + b * T) - Tm
        acc = acc + c[j] * Tn
        Tm, T = T, Tn
    return acc


def power_method(apply_H, v0, iters=50):
    """Largest eigenvalue estimate of a Hermitian PSD H by the power method
    (used for the upper Chebyshev bound, Sec. 2.3 and Sec. 3)."""
    v = np.asarray(v0, dtype=np.complex128)
    v = v / np.linalg.norm(v)
    lam = 0.0
    for _ in range(iters):
        w = apply_H(v)
        lam = float(np.vdot(v, w).real)
        v = w / np.linalg.norm(w)
    return lam


def lanczos_extremes(apply_H, v0, steps):
    """Extreme Ritz values of a Hermitian H after ``steps`` Lanczos steps (no
    reorthogonalisation; extreme Ritz values are unaffected by the loss of
    orthogonality).  Returns (theta_min, theta_max, bound_min, bound_max)
    where bound = |beta_k * last component of the Ritz vector| bounds the
    distance of theta to the nearest eigenvalue."""
    v = np.asarray(v0, dtype=np.complex128).reshape(-1)
    v = v / np.linalg.norm(v)
    v_prev = np.zeros_like(v)
    alphas, betas = [], []
    beta = 0.0
    for _ in range(steps):
        w = apply_H(v).reshape(-1)
        alpha = float(np.vdot(v, w).real)
        w = w - alpha * v - beta * v_prev
        beta = float(np.linalg.norm(w))
        alphas.append(alpha)
        betas.append(beta)
        if beta == 0.0:
            break
        v_prev, v = v, w / beta
    k = len(alphas)
    Tk = np.diag(alphas) + np.diag(betas[:k - 1], 1) + np.diag(betas[:k - 1], -1)
    evals, evecs = np.linalg.eigh(Tk)
    bmin = abs(betas[-1] * evecs[-1, 0])
    bmax = abs(betas[-1] * evecs[-1, -1])
    return float(evals[0]), float(evals[-1]), float(bmin), float(bmax)


def cg5d(apply_H, B, X0=None, tol=1e-10, maxiter=1000, history=None):
    """Conjugate gradients on the enlarged system (Sec. 2.1: the coarse solve
    treated as one five-dimensional system with a single Krylov space, block
    diagonal in the right-hand-side index).  The vector is the whole block
    [V][nb][R]; alpha and beta come from inner products summed over all
    right-hand sides; the iteration stops when every column's recurrence
    residual satisfies |r_j| <= tol |b_j|, and the result carries the true
    residuals."""
    shape = B.shape
    Bm = as_matrix(np.asarray(B, dtype=np.complex128))
    R = Bm.shape[1]
    H = lambda M: as_matrix(apply_H(M.reshape(shape)))
    X = np.zeros_like(Bm) if X0 is None else as_matrix(np.asarray(X0, dtype=np.complex128)).copy()
    r = Bm - H(X)
    p = r.copy()
    rr = np.vdot(r, r).real
    bn = np.linalg.norm(Bm, axis=0)
    k = 0
    for k in range(1, maxiter + 1):
        w = H(p)
        alpha = rr / np.vdot(p, w).real
        X = X + alpha * p
        r = r - alpha * w
        rr_new = np.vdot(r, r).real
        if history is not None:
            history.append(dict(X=X.copy(), r=r.copy(), alpha=alpha))
        if np.all(np.linalg.norm(r, axis=0) <= tol * np.where(bn > 0, bn, 1.0)):
            break
        p = r + (rr_new / rr) * p
        rr = rr_new
    res = np.linalg.norm(Bm - H(X), axis=0) / np.where(bn > 0, bn, 1.0)
    return X.reshape(shape), dict(iters=k, resid=res)
