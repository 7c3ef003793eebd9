"""The decomposed coarse solve (Sec. 2.6 ghost-zone exchange, Fig. 2 left
with Grams summed over ranks) on CPU ranks over gloo.

Each rank runs the product's host side -- paper_2409_03904_b300.domain:
geometry, the dimension-by-dimension halo exchange and the sharded
BlockCGrQ iteration -- with a CPU backend built here from the oracle in
place of the library's CUDA kernels (rows copied with numpy indexing, the
local operator evaluated from its own neighbour table, Grams, block
updates and Cholesky factors from oracle/).  The sharded operator and the
sharded solve must equal the oracle's operator and its BlockCGrQ on the
whole lattice: world size 2 (one dimension cut) and world size 4 (two
dimensions cut, so the 81-point stencil's corner sites must travel through
the first exchange's ghost layers).
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle.chol import chol_upper, hermitian_part, upper_inverse
from oracle.ops import block_axpy, block_inner, coarse_op_apply
from oracle.solvers import block_cg_rq
from synth import coarse_op, stencil, vectors


class OracleBackend:
    """CPU stand-in for domain.DeviceBackend: the same calls, computed with
    numpy and the oracle on torch CPU tensors (gloo moves those)."""

    def __init__(self, dom, A_local, disp):
        self.dom, self.A, self.nb = dom, A_local, A_local.shape[2]
        # the local operator's input sites, from coordinates: owned site c
        # reads c + h + delta on the padded lattice, wrapping periodically
        # only where there is no ghost layer
        l, Lin, h = np.array(dom.l), np.array(dom.Lin), np.array(dom.h)
        x = np.arange(dom.V)
        c = np.stack([(x // np.prod(l[:mu])) % l[mu] for mu in range(4)], axis=-1)
        self.nbr = []
        for d in np.asarray(disp, dtype=np.int64):
            y = np.mod(c + h + d, Lin)
            self.nbr.append(y[:, 0] + Lin[0] * (y[:, 1] + Lin[1] * (y[:, 2] + Lin[2] * y[:, 3])))
        self._pad = {}

    def zeros_like(self, X):
        return torch.zeros_like(X)

    def empty_like(self, X):
        return torch.zeros_like(X)

    def copy(self, X):
        return X.clone()

    def copy_into(self, Y, X):
        Y.copy_(X)
        return Y

    def padded(self, R):
        if R not in self._pad:
            self._pad[R] = torch.zeros((self.dom.Vin, self.nb, R), dtype=torch.complex128)
        return self._pad[R]

    def gather(self, Xpad, idx):
        return Xpad[torch.from_numpy(idx)].clone()

    def scatter(self, buf, idx, Xpad):
        Xpad[torch.from_numpy(idx)] = buf
        return Xpad

    def apply(self, Xpad):
        X = Xpad.numpy()
        Y = np.zeros((self.dom.V, self.nb, X.shape[-1]), dtype=np.complex128)
        for p, nbr in enumerate(self.nbr):
            Y += np.matmul(self.A[:, p], X[nbr])
        return torch.from_numpy(Y)

    def gram(self, X, Y):
        return torch.from_numpy(block_inner(X.numpy(), Y.numpy()))

    def axpy(self, Y, X, M, beta):
        Y.copy_(torch.from_numpy(np.ascontiguousarray(
            block_axpy(Y.numpy(), X.numpy(), M.numpy(), beta).reshape(Y.shape))))
        return Y

    def mm(self, A, B):
        return torch.from_numpy(A.numpy() @ B.numpy())

    def adj(self, A):
        return torch.from_numpy(np.ascontiguousarray(np.conj(A.numpy().T)))

    def eye(self, R, a):
        return a * torch.eye(R, dtype=torch.complex128)

    def factor(self, G, tau):
        S = chol_upper(hermitian_part(G.numpy()), tau)
        return torch.from_numpy(S), torch.from_numpy(upper_inverse(S)), S.shape[0]

    def diag(self, G):
        return np.real(np.diag(G.numpy())).copy()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _worker(rank, world, port, grid, L, nb, npts, R, shift):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    torch.set_num_threads(1)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2409_03904_b300 import domain
        disp, _ = stencil(npts)
        A = coarse_op(L, nb, npts, 4040, shift)
        B = vectors(L, nb, R, 4041)
        dom = domain.Domain(L, grid, rank)
        gs = dom.global_sites
        be = OracleBackend(dom, A[gs], disp)
        comm = domain.TorchComm()
        # the sharded operator on this rank's sites
        Y = domain.apply(dom, be, torch.from_numpy(B[gs].copy()), comm).numpy()
        Yref = coarse_op_apply(A, B, L, disp)[gs]
        assert _rel(Y, Yref) <= 1e-13, ("operator", rank, _rel(Y, Yref))
        # the sharded BlockCGrQ against the oracle's on the whole lattice
        X, info = domain.block_cg(dom, be, comm, torch.from_numpy(B[gs].copy()), tol=1e-10,
                                  maxiter=400)
        Xo, io = block_cg_rq(lambda V: coarse_op_apply(A, V, L, disp), B, tol=1e-10, maxiter=400)
        assert io["converged"] and info["converged"], (info, io)
        assert abs(info["iters"] - io["iters"]) <= 1, (info["iters"], io["iters"])
        assert _rel(X.numpy(), Xo[gs]) <= 1e-9, ("solve", rank, _rel(X.numpy(), Xo[gs]))
        assert max(info["resid"]) <= 1e-10
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("grid,npts", [((1, 1, 1, 2), 81), ((1, 1, 2, 2), 81), ((2, 1, 1, 1), 9)])
def test_decomposed_operator_and_block_cg(grid, npts):
    world = int(np.prod(grid))
    L, nb, R = (4, 3, 4, 4), 4, 3
    mp.spawn(_worker, args=(world, _free_port(), grid, L, nb, npts, R, 40.0), nprocs=world,
             join=True)


def test_domain_geometry():
    """Faces and ghost layers: on a rank grid of 2 along the last dimension,
    each rank owns half the lattice; its ghost layers hold exactly the global
    sites one step beyond its owned block, and its send faces are its first
    and last owned layers (with all padded sites of the other dimensions)."""
    from paper_2409_03904_b300 import domain
    L, grid = (4, 3, 4, 4), (1, 1, 1, 2)
    for rank in range(2):
        dom = domain.Domain(L, grid, rank)
        assert dom.l == (4, 3, 4, 2) and dom.h == (0, 0, 0, 1) and dom.Lin == (4, 3, 4, 4)
        assert dom.minus[3] == dom.plus[3] == 1 - rank
        f = dom.faces[3]
        for key, c3 in (("send_lo", 1), ("send_hi", 2), ("recv_lo", 0), ("recv_hi", 3)):
            idx = f[key]
            assert len(idx) == 4 * 3 * 4
            assert np.all(idx // (4 * 3 * 4) == c3)
        # owned sites tile the lattice across ranks
    owned = np.concatenate([domain.Domain(L, grid, r).global_sites for r in range(2)])
    assert np.array_equal(np.sort(owned), np.arange(int(np.prod(L))))
    with pytest.raises(ValueError):
        domain.Domain(L, (1, 2, 1, 1), 0)        # 2 does not divide 3


class FailingComm:
    """A rank that fails between steps: its `fail_at`-th Gram allreduce raises
    instead of taking part. This is the host-side form of a rank that crashes
    (no GPU work is in flight at that point)."""

    def __init__(self, inner, fail_at):
        self.inner, self.calls, self.fail_at = inner, 0, fail_at

    def allreduce(self, t):
        self.calls += 1
        if self.calls == self.fail_at:
            raise RuntimeError("injected rank failure")
        return self.inner.allreduce(t)

    def sendrecv(self, *args):
        return self.inner.sendrecv(*args)


def _failing_worker(rank, world, port, grid, L, nb, npts, R, shift, q):
    import datetime
    import time
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    torch.set_num_threads(1)
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=20))
    t0 = time.time()
    outcome = "finished"
    try:
        from paper_2409_03904_b300 import domain
        disp, _ = stencil(npts)
        A = coarse_op(L, nb, npts, 4040, shift)
        B = vectors(L, nb, R, 4041)
        dom = domain.Domain(L, grid, rank)
        gs = dom.global_sites
        be = OracleBackend(dom, A[gs], disp)
        comm = domain.TorchComm()
        if rank == 1:
            comm = FailingComm(comm, fail_at=5)
        domain.block_cg(dom, be, comm, torch.from_numpy(B[gs].copy()), tol=1e-10, maxiter=400)
    except Exception as e:  # noqa: BLE001  (every outcome is reported to the parent)
        outcome = f"{type(e).__name__}: {str(e)[:200]}"
    q.put((rank, outcome, time.time() - t0))
    q.close()
    q.join_thread()
    if rank == 1:
        os._exit(0)          # the failed rank leaves without a clean shutdown
    try:
        dist.destroy_process_group()
    except Exception:  # noqa: BLE001
        pass


def test_rank_failure_ends_the_other_ranks_solve():
    """A rank of the decomposed BlockCGrQ fails between iterations and exits.
    The other rank must not hang: its next collective raises, within the
    process group's 20 s timeout. Plain spawned processes report through a
    queue, so the harness does not kill the survivor before it detects the
    failure."""
    import multiprocessing
    ctx = multiprocessing.get_context("spawn")
    q = ctx.Queue()
    L, nb, R = (4, 3, 4, 4), 4, 3
    port = _free_port()
    procs = [ctx.Process(target=_failing_worker,
                         args=(r, 2, port, (1, 1, 1, 2), L, nb, 81, R, 40.0, q))
             for r in range(2)]
    for p in procs:
        p.start()
    res = {}
    try:
        for _ in range(2):
            r, outcome, dt = q.get(timeout=120)
            res[r] = (outcome, dt)
    finally:
        for p in procs:
            p.join(timeout=30)
            if p.is_alive():
                p.kill()
    assert "injected rank failure" in res[1][0], res
    assert res[0][0] != "finished", res            # the survivor's collective failed
    assert res[0][1] < 60, res                     # and it did not wait forever
    print("survivor:", res[0])
