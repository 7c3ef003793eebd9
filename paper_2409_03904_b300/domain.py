"""The coarse solve on a 4D-decomposed lattice, one rank per GPU.

Sec. 2.6 ("Applying the coarse operator") describes the distributed coarse
operator: every rank owns a block of the lattice and the coefficients of its
sites; the input vector of an application lives on the padded local volume,
whose ghost layers are filled by a halo exchange done one dimension after the
other, each exchange carrying the ghost layers of the dimensions before it,
so the corner sites of the 81-point stencil arrive through nearest-neighbour
messages only; the result lives on the owned sites.  The block CG of Fig. 2
(left) then needs one more collective: every nrhs x nrhs Gram is a sum over
all sites, i.e. a local Gram followed by an allreduce.

This module is the host side of that scheme:

* ``Domain``: the geometry -- owned extents, the rank grid, the neighbour
  ranks, and, per padded dimension, the padded-site indices of the faces to
  send and of the ghost layers to fill (integer bookkeeping only);
* ``exchange_halo``: the dimension-by-dimension ghost-zone exchange
  (faces gathered into buffers, messages swapped with the two neighbours,
  buffers scattered into the ghost layers);
* ``apply``: owned X -> padded input -> exchange -> local operator;
* ``block_cg``: BlockCGrQ (Fig. 2 left, X update carrying C_k) with every
  Gram summed over ranks.

The arithmetic runs in a *backend*; ``DeviceBackend`` calls the library's
kernels (mrhs_op_create_halo operator, block_inner, block_axpy, herm_factor,
mrhs_gather_rows / mrhs_scatter_rows) on the current CUDA device.  Messages
and the Gram allreduce go through ``TorchComm`` (torch.distributed: NCCL
between GPUs).  The degenerate rank grid (1, 1, 1, 1) with a forced ghost
layer exchanges with itself and runs on one GPU.

Limits: the lattice extents must be divisible by the rank grid; every
right-hand side must be nonzero and the block must keep full rank until
convergence (the single-GPU block_cg_solve also handles zero columns and
rank loss); operators with a halo are built in FP64, DF32, FP32 or OZ.
"""
import ctypes
import math

import numpy as np
import torch

from . import _lib


def _coords(idx, ext):
    """Coordinates (first dimension fastest) of site indices on extents ext."""
    idx = np.asarray(idx, dtype=np.int64)
    out = []
    for e in ext:
        out.append(idx % e)
        idx = idx // e
    return np.stack(out, axis=-1)


def _index(c, ext):
    c = np.asarray(c, dtype=np.int64)
    return c[..., 0] + ext[0] * (c[..., 1] + ext[1] * (c[..., 2] + ext[2] * c[..., 3]))


class Domain:
    """One rank's block of the periodic lattice L on the rank grid P.

    Rank r has grid coordinates q (first dimension fastest, like sites) and
    owns the sites with global coordinates q * l + c, c in [0, l), l = L / P.
    A dimension with P > 1 (or forced by ``pad``) gets a ghost layer of depth
    one on both sides; in the others the local lattice wraps periodically
    (it is the whole extent).
    """

    def __init__(self, L, grid, rank, pad=(0, 0, 0, 0)):
        self.L = tuple(int(v) for v in L)
        self.P = tuple(int(v) for v in grid)
        if len(self.L) != 4 or len(self.P) != 4:
            raise ValueError("L and grid need four extents")
        for a, p in zip(self.L, self.P):
            if p < 1 or a % p:
                raise ValueError(f"rank grid {self.P} does not divide the lattice {self.L}")
        self.size = int(np.prod(self.P))
        if not 0 <= rank < self.size:
            raise ValueError("rank outside the grid")
        self.rank = int(rank)
        self.q = tuple(int(v) for v in _coords(self.rank, self.P))
        self.l = tuple(a // p for a, p in zip(self.L, self.P))
        self.h = tuple(1 if (p > 1 or pd) else 0 for p, pd in zip(self.P, pad))
        self.Lin = tuple(a + 2 * h for a, h in zip(self.l, self.h))
        self.V = int(np.prod(self.l))
        self.Vin = int(np.prod(self.Lin))
        c = _coords(np.arange(self.V), self.l)
        # padded index of each owned site, and its global site index
        self.interior = _index(c + np.asarray(self.h), self.Lin)
        self.global_sites = _index(c + np.asarray(self.q) * np.asarray(self.l), self.L)
        # neighbour ranks in each dimension
        self.minus, self.plus = [], []
        for mu in range(4):
            qm, qp = list(self.q), list(self.q)
            qm[mu] = (qm[mu] - 1) % self.P[mu]
            qp[mu] = (qp[mu] + 1) % self.P[mu]
            self.minus.append(int(_index(np.asarray(qm), self.P)))
            self.plus.append(int(_index(np.asarray(qp), self.P)))
        # faces of each padded dimension: every padded site with the given
        # coordinate in mu (all padded coordinates in the other dimensions, so
        # the ghost layers of earlier dimensions travel along), ordered by
        # padded site index -- the same order on every rank
        cp = _coords(np.arange(self.Vin), self.Lin)
        self.faces = {}
        for mu in range(4):
            if not self.h[mu]:
                continue
            n = self.Lin[mu]
            at = lambda v: np.nonzero(cp[:, mu] == v)[0].astype(np.int64)  # noqa: E731
            self.faces[mu] = dict(send_lo=at(1), send_hi=at(n - 2), recv_lo=at(0),
                                  recv_hi=at(n - 1))

    def local_part(self, X):
        """Rows of a global [V][...] array that this rank owns."""
        return X[self.global_sites]


class TorchComm:
    """Messages and sums between ranks through torch.distributed."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group

    def allreduce(self, t):
        self.dist.all_reduce(t, group=self.group)
        return t

    def sendrecv(self, mu, lo, hi, minus, plus):
        """Send the low face to the minus neighbour and the high face to the
        plus neighbour; receive the plus neighbour's low face (our high ghost
        layer) and the minus neighbour's high face (our low ghost layer).
        Tags 2 mu / 2 mu + 1 keep the two messages apart when both
        neighbours are the same rank."""
        d = self.dist
        rlo, rhi = torch.empty_like(hi), torch.empty_like(lo)
        ops = [d.P2POp(d.isend, lo.contiguous(), minus, self.group, 2 * mu),
               d.P2POp(d.isend, hi.contiguous(), plus, self.group, 2 * mu + 1),
               d.P2POp(d.irecv, rhi, plus, self.group, 2 * mu),
               d.P2POp(d.irecv, rlo, minus, self.group, 2 * mu + 1)]
        for w in d.batch_isend_irecv(ops):
            w.wait()
        return rlo, rhi


class SelfComm:
    """A world of one rank: sums are the local values."""

    def allreduce(self, t):
        return t

    def sendrecv(self, mu, lo, hi, minus, plus):
        raise RuntimeError("a one-rank world has no neighbours")


def exchange_halo(dom, Xpad, be, comm):
    """Fill the ghost layers of the padded vector Xpad, dimension after
    dimension (Sec. 2.6)."""
    for mu in range(4):
        if not dom.h[mu]:
            continue
        f = dom.faces[mu]
        lo = be.gather(Xpad, f["send_lo"])
        hi = be.gather(Xpad, f["send_hi"])
        if dom.minus[mu] == dom.rank:          # P[mu] == 1: the periodic wrap is local
            rlo, rhi = hi, lo
        else:
            rlo, rhi = comm.sendrecv(mu, lo, hi, dom.minus[mu], dom.plus[mu])
        be.scatter(rlo, f["recv_lo"], Xpad)
        be.scatter(rhi, f["recv_hi"], Xpad)
    return Xpad


def apply(dom, be, X, comm):
    """Y = H X on the owned sites: owned rows into the padded buffer, ghost
    layers exchanged, the local operator applied."""
    Xpad = be.padded(X.shape[-1])
    be.scatter(X, dom.interior, Xpad)
    exchange_halo(dom, Xpad, be, comm)
    return be.apply(Xpad)


def block_cg(dom, be, comm, B, tol=1e-8, maxiter=1000, X0=None, tau=1e-14):
    """BlockCGrQ (Fig. 2 left) for H X = B on the decomposed lattice.

    Every rank passes its owned rows of B (and X0) and receives its rows of
    X; the small nrhs x nrhs algebra is replicated (every rank factors the
    same summed Gram).  Readings: X_{k+1} = X_k + D_k M_k C_k; the Grams are
    Hermitian-symmetrised before their factorisation; stop when every
    column's recurrence estimate |C e_r| <= tol |b_r|, then report the true
    residuals.  Returns (X, info)."""
    R = int(B.shape[-1])
    bn = np.sqrt(be.diag(comm.allreduce(be.gram(B, B))))
    if not np.all(bn > 0):
        raise ValueError("block_cg: every right-hand side must be nonzero")
    H = lambda V: apply(dom, be, V, comm)  # noqa: E731
    if X0 is None:
        X = be.zeros_like(B)
        Rk = be.copy(B)
    else:
        X = be.copy(X0)
        Rk = be.axpy(be.copy(B), H(X), be.eye(R, -1.0), 1.0)
    S, W = _factor(be, comm.allreduce(be.gram(Rk, Rk)), R, tau)
    C = S                                                     # R_0 = Q_0 C_0
    Q = be.axpy(be.empty_like(B), Rk, W, 0.0)
    D = be.copy(Q)
    T = be.empty_like(B)
    k, converged = 0, False
    for k in range(1, maxiter + 1):
        Z = H(D)                                              # Z_k = H D_k
        S1, W1 = _factor(be, comm.allreduce(be.gram(D, Z)), R, tau)
        M = be.mm(W1, be.adj(W1))                             # [D^dag Z]^-1
        be.axpy(X, D, be.mm(M, C), 1.0)                       # X + D M C
        be.copy_into(T, Q)
        be.axpy(T, Z, be.mm(M, be.eye(R, -1.0)), 1.0)         # T = Q - Z M
        S, W = _factor(be, comm.allreduce(be.gram(T, T)), R, tau)
        be.axpy(Q, T, W, 0.0)                                 # Q_{k+1} = T S^-1
        be.axpy(T, D, be.adj(S), 0.0)                         # D S^dag
        be.copy_into(D, Q)
        be.axpy(D, T, be.eye(R, 1.0), 1.0)                    # D = Q + D S^dag
        C = be.mm(S, C)                                       # C_{k+1} = S C
        est = np.sqrt(be.diag(be.gram(C, C))) / bn            # |C e_r| / |b_r|
        if np.all(est <= tol):
            converged = True
            break
    r = be.axpy(be.copy(B), H(X), be.eye(R, -1.0), 1.0)
    res = np.sqrt(be.diag(comm.allreduce(be.gram(r, r)))) / bn
    return X, dict(iters=k, converged=bool(converged and np.all(res <= 10 * tol)),
                   resid=[float(v) for v in res])


def _factor(be, G, R, tau):
    S, W, rank = be.factor(G, tau)
    if rank < R:
        raise _lib.MrhsError(-4, f"block_cg: the block lost rank ({rank} of {R})")
    return S, W


class DeviceBackend:
    """The block algebra and the local operator on the current CUDA device,
    through the library's kernels.  ``op`` is the rank's CoarseOp with the
    domain's halo (mrhs_op_create_halo) and ``prec`` its FP64 precision
    ("fp64" or "oz")."""

    def __init__(self, dom, op, prec="fp64"):
        self.dom, self.op, self.prec = dom, op, prec
        self.nb = op.nb
        self.dev = op.device
        self._idx = {}
        self._pad = {}
        self.lib = _lib.lib()

    # ---- vectors [sites][nb][R] complex128
    def zeros_like(self, X):
        return torch.zeros_like(X)

    def empty_like(self, X):
        return torch.empty_like(X)

    def copy(self, X):
        return X.clone()

    def copy_into(self, Y, X):
        Y.copy_(X)
        return Y

    def padded(self, R):
        if R not in self._pad:
            self._pad[R] = torch.zeros((self.dom.Vin, self.nb, R), dtype=torch.complex128,
                                       device=self.dev)
        return self._pad[R]

    def _dev_idx(self, idx):
        key = id(idx)
        if key not in self._idx:
            self._idx[key] = (idx, torch.from_numpy(np.ascontiguousarray(idx)).to(self.dev))
        return self._idx[key][1]

    def gather(self, Xpad, idx):
        rb = Xpad[0].numel() * Xpad.element_size()
        buf = torch.empty((len(idx),) + tuple(Xpad.shape[1:]), dtype=Xpad.dtype, device=self.dev)
        _lib.check(self.lib.mrhs_gather_rows(_lib.dev_ptr(Xpad), Xpad.shape[0],
                                             _lib.dev_ptr(self._dev_idx(idx)), len(idx),
                                             _lib.dev_ptr(buf), rb, _lib.stream_ptr()))
        return buf

    def scatter(self, buf, idx, Xpad):
        rb = Xpad[0].numel() * Xpad.element_size()
        buf = buf.to(self.dev).contiguous()
        _lib.check(self.lib.mrhs_scatter_rows(_lib.dev_ptr(buf), len(idx),
                                              _lib.dev_ptr(self._dev_idx(idx)), _lib.dev_ptr(Xpad),
                                              Xpad.shape[0], rb, _lib.stream_ptr()))
        return Xpad

    def apply(self, Xpad):
        return self.op.apply(Xpad, self.prec)

    # ---- nrhs x nrhs algebra (device complex128)
    def gram(self, X, Y):
        from . import block_inner
        return block_inner(X, Y)

    def axpy(self, Y, X, M, beta):
        from . import block_axpy
        return block_axpy(Y, X, M, beta)

    def mm(self, A, B):
        """A B for small square matrices: a block update with A's rows as
        the 'sites' (block_axpy on an R-row block)."""
        from . import block_axpy
        out = torch.empty((A.shape[0], B.shape[1]), dtype=torch.complex128, device=self.dev)
        return block_axpy(out, A.contiguous(), B, 0.0)

    def adj(self, A):
        """A^dagger as the Gram A^dagger I (block_inner)."""
        from . import block_inner
        return block_inner(A.contiguous(), self.eye(A.shape[0], 1.0))

    def eye(self, R, a):
        key = ("eye", R, a)
        if key not in self._pad:
            self._pad[key] = (a * torch.eye(R, dtype=torch.complex128)).to(self.dev)
        return self._pad[key]

    def factor(self, G, tau):
        from . import herm_factor
        return herm_factor(G, tau)

    def diag(self, G):
        """The real diagonal of a small device matrix, read back to the host
        (the stopping test)."""
        return G.diagonal().real.cpu().numpy()


def halo_op(dom, A_local, disp, precisions=("fp64",)):
    """The rank's operator: its owned sites' coefficients with the domain's
    ghost layers (mrhs_op_create_halo)."""
    from . import CoarseOp
    return CoarseOp(A_local, dom.l, disp, precisions, halo=dom.h)
