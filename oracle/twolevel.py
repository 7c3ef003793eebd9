"""Two-level ADEF2 preconditioner and the flexible ADEF2 conjugate gradient of
Fig. 1, complex128.

Test infrastructure only (see the package docstring).

Fig. 1 and Sec. 2 ("Multigrid and the HDCG algorithm"):
* coarse-grid correction Q = P h^-1 P^dagger, with P the blocked basis
  (promote), P^dagger its adjoint (project) and h = P^dagger H P the coarse
  operator (little Dirac operator, Eq. coarseop); in the paper's block
  notation Q = diag(0, H_SS^-1);
* P_R = I - Q H (the Petrov-Galerkin projector of Sec. 2, written there as
  L^-1 P_Sbar);
* preconditioner M^-1 = P_R S + Q with S the smoother M_IRS(H, Lambda),
  applied as t + Q (r - H t) with t = S r (identical for a linear Q; the
  reading for the variable coarse solve, see adef2_apply);
* start x_0 = Q b + P_R x for an arbitrary x;
* the flexible CG iteration of Fig. 1.

Readings of Fig. 1 (the figure is terse and in two places garbled):
* step 9 divides (r_k, y_k) by (p_k, w_k); y_k appears nowhere else and is
  read as z_k, the preconditioned residual of step 5 / step 12;
* step 8 orthogonalises the new search direction against the last m_max
  ones.  Its coefficient, printed as (d_k, H w_i)/(w_i, H w_i), is read as
  the H-inner-product projection of flexible CG (Notay 2000; the paper
  cites "flexible CG" for this step): c_i = (p_i, d_k)/(p_i, w_i) with
  d_k = H p_k and w_i = H p_i, applied to both the direction,
  p_k <- p_k - c_i p_i, and its image, w_k = d_k - sum_i c_i w_i, so that
  w_k = H p_k still holds and r_{k+1} = r_k - alpha_k w_k remains the true
  residual recurrence;
* several right-hand sides run as independent single-vector processes (the
  paper runs its smoother and its flexible outer solve per right-hand side).

The variable (Krylov) preconditioner of the original HDCG is
  S = a fixed number of CG iterations on H + Lambda (the infra-red shift
      smoother, N_cg = 7, Lambda = 2 in the paper), and
  h^-1 = deflated CG to a loose residual (4e-2 in the paper), read here as
      CG started from the deflated guess U Lambda_ev^-1 U^dagger b;
the stationary one of Sec. 2.3 is
  S = the Chebyshev approximation to 1/x (order 8 on [2, hi] in the paper),
  h^-1 = Q^{Cheby+defl} (oracle.deflation.defl_cheby_apply).
"""
import numpy as np

from .ops import as_matrix


def coarse_correction(project, promote, coarse_solve, r):
    """Q r = P h^-1 P^dagger r."""
    return promote(coarse_solve(project(r)))


def adef2_apply(apply_H, smoother, coarse, r):
    """M^-1 r = P_R S r + Q r (Fig. 1, step 2) with P_R = 1 - Q H, evaluated
    as t + Q (r - H t), t = S r: one coarse solve on the smoothed residual.
    For a linear Q this is S r - Q H S r + Q r exactly; for the variable
    (Krylov) coarse solve the figure's sum is read this way, the form a
    two-level cycle takes (``coarse`` applies Q)."""
    t = smoother(r)
    return t + coarse(r - apply_H(t))


def cg_fixed(apply_H, b, iters):
    """``iters`` iterations of plain CG from x = 0 for one right-hand side
    (the fixed-iteration smoother M_IRS); an iteration whose residual has
    vanished ends early."""
    b = np.asarray(b, dtype=np.complex128)
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rr = np.vdot(r, r).real
    for _ in range(iters):
        if rr == 0.0:
            break
        w = apply_H(p)
        alpha = rr / np.vdot(p, w).real
        x = x + alpha * p
        r = r - alpha * w
        rr_new = np.vdot(r, r).real
        p = r + (rr_new / rr) * p
        rr = rr_new
    return x


def cg_to_tol(apply_H, b, x0, tol, maxiter):
    """Plain CG from x0 until |b - H x| <= tol |b| (recurrence residual) or
    maxiter iterations."""
    b = np.asarray(b, dtype=np.complex128)
    x = np.asarray(x0, dtype=np.complex128).copy()
    r = b - apply_H(x)
    p = r.copy()
    rr = np.vdot(r, r).real
    bn = np.linalg.norm(b)
    for _ in range(maxiter):
        if np.sqrt(rr) <= tol * bn:
            break
        w = apply_H(p)
        alpha = rr / np.vdot(p, w).real
        x = x + alpha * p
        r = r - alpha * w
        rr_new = np.vdot(r, r).real
        p = r + (rr_new / rr) * p
        rr = rr_new
    return x


def deflated_guess(U, lam, b):
    """U Lambda^-1 U^dagger b for orthonormal eigenvectors U (columns)."""
    return U @ ((np.conj(U).T @ b) / np.asarray(lam, dtype=np.float64))


def flex_adef2(apply_H, apply_Minv, coarse, b, x=None, tol=1e-8, maxiter=1000, mmax=1,
               history=None):
    """Flexible ADEF2 preconditioned CG (Fig. 1) for one right-hand side b.

    apply_Minv: the preconditioner M^-1 (possibly variable); coarse: Q (for
    the start x_0 = Q b + P_R x).  Returns (x, info) with info = {iters,
    resid (true, relative), converged}."""
    b = np.asarray(b, dtype=np.complex128).reshape(-1)
    xa = np.zeros_like(b) if x is None else np.asarray(x, dtype=np.complex128).reshape(-1)
    # x_0 = Q b + P_R x = Q b + x - Q H x
    x = coarse(b) + xa - coarse(apply_H(xa))
    r = b - apply_H(x)
    bn = np.linalg.norm(b)
    if np.linalg.norm(r) <= tol * bn:                       # the start already solves it
        return x, dict(iters=0, resid=float(np.linalg.norm(r) / bn), converged=True)
    z = apply_Minv(r)
    p = z.copy()
    rz = np.vdot(r, z)
    hist = []
    k = 0
    converged = False
    for k in range(1, maxiter + 1):
        d = apply_H(p)                                      # d_k = H p_k
        w = d.copy()
        for pi, wi in hist[-mmax:] if mmax > 0 else []:     # step 8 (reading above)
            c = np.vdot(pi, d) / np.vdot(pi, wi)
            p = p - c * pi
            w = w - c * wi
        alpha = rz / np.vdot(p, w)                          # (r_k, z_k)/(p_k, w_k)
        x = x + alpha * p
        r = r - alpha * w
        hist.append((p.copy(), w.copy()))
        if history is not None:
            history.append(dict(x=x.copy(), r=r.copy(), p=p.copy(), w=w.copy()))
        if np.linalg.norm(r) <= tol * bn:
            converged = True
            break
        z = apply_Minv(r)
        rz_new = np.vdot(r, z)
        beta = rz_new / rz
        p = z + beta * p
        rz = rz_new
    res = np.linalg.norm(b - apply_H(x)) / bn
    return x, dict(iters=k, resid=float(res), converged=bool(converged and res <= 10 * tol))


def flex_adef2_columns(apply_H, apply_Minv, coarse, B, tol=1e-8, maxiter=1000, mmax=1):
    """flex_adef2 on every column of B ([N][R] or [V][nb][R]) independently;
    apply_H / apply_Minv / coarse act on single vectors of N entries."""
    Bm = as_matrix(np.asarray(B, dtype=np.complex128))
    X = np.zeros_like(Bm)
    infos = []
    for j in range(Bm.shape[1]):
        X[:, j], info = flex_adef2(apply_H, apply_Minv, coarse, Bm[:, j], tol=tol,
                                   maxiter=maxiter, mmax=mmax)
        infos.append(info)
    return X.reshape(np.shape(B)), infos
