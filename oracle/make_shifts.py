"""Write tests/golden/shifts.json: the self-term shift c of every named workload.

Test infrastructure only (see the package docstring).  Run as
    python -m oracle.make_shifts [name ...] [--steps K] [--procs P]

Input recipe: the unshifted Hermitian operator H0 (c = 0) is generated from
the seeded recipe in ``synth``; its extreme eigenvalues lam_min, lam_max are
estimated (dense eigvalsh up to N = 8192, otherwise Lanczos with the C
oracle operator on the self and positive-displacement blocks); then
    c = (lam_max - kappa * lam_min) / (kappa - 1)
so that (lam_max + c) / (lam_min + c) = kappa.  Lanczos Ritz values lie
inside the spectrum, so the record carries each one's residual bound, and
the Gershgorin radius of H0 for reference.
"""
import argparse
import json
import multiprocessing as mp
import os
import sys
import time
from multiprocessing import shared_memory

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
OUT = os.path.join(ROOT, "tests", "golden", "shifts.json")


def _positive_points(npts):
    from synth import stencil
    from synth.coarse import is_positive
    disp, _ = stencil(npts)
    pos = [p for p in range(1, npts) if is_positive(tuple(int(v) for v in disp[p]))]
    return disp, pos


def _gen_chunk(args):
    shm_name, shape, L, nb, npts, seed, points, s0, s1 = args
    from synth import coarse_op
    shm = shared_memory.SharedMemory(name=shm_name)
    try:
        arr = np.ndarray(shape, dtype=np.complex128, buffer=shm.buf)
        arr[s0:s1] = coarse_op(L, nb, npts, seed, 0.0, sites=np.arange(s0, s1), points=points)
    finally:
        shm.close()
    return s1 - s0


def generate_half(L, nb, npts, seed, procs):
    """Self + positive-displacement blocks of H0, [V][1 + npos][nb][nb]."""
    disp, pos = _positive_points(npts)
    points = [0] + pos
    V = int(np.prod(L))
    shape = (V, len(points), nb, nb)
    nbytes = int(np.prod(shape)) * 16
    shm = shared_memory.SharedMemory(create=True, size=nbytes)
    chunk = max(1, V // (procs * 8))
    jobs = [(shm.name, shape, L, nb, npts, seed, points, s, min(V, s + chunk))
            for s in range(0, V, chunk)]
    if procs > 1:
        with mp.get_context("spawn").Pool(procs) as pool:
            for _ in pool.imap_unordered(_gen_chunk, jobs):
                pass
    else:
        for j in jobs:
            _gen_chunk(j)
    # no copy: the largest lattice fills half of the host memory on its own;
    # the caller releases the block with release_half()
    out = np.ndarray(shape, dtype=np.complex128, buffer=shm.buf)
    _LIVE[id(out)] = shm
    return out, disp[pos]


_LIVE = {}


def release_half(arr):
    shm = _LIVE.pop(id(arr), None)
    del arr
    if shm is not None:
        shm.close()
        shm.unlink()


def gershgorin_radius(Ahalf):
    """max_x,a sum_b |row| over all blocks of a row (each hop block appears
    once as A_p(x) and once as a conjugate-transposed partner in some row;
    the bound uses 2x the positive blocks' row sums, an upper bound)."""
    best = 0.0
    for s0 in range(0, Ahalf.shape[0], 1024):     # site chunks: bounded temporaries
        blk = np.abs(Ahalf[s0:s0 + 1024])
        rows = blk[:, 0].sum(axis=-1) + blk[:, 1:].sum(axis=(1, 3)) + blk[:, 1:].sum(axis=(1, 2))
        best = max(best, float(rows.max()))
    return best


def estimate(w, steps, procs):
    from oracle import native
    from oracle.solvers import lanczos_extremes
    from synth import vectors
    L, nb, npts, seed, kappa = w["L"], w["nb"], w["npts"], w["seed"], w["kappa"]
    t0 = time.time()
    Ahalf, pos_disp = generate_half(L, nb, npts, seed, procs)
    tgen = time.time() - t0
    N = int(np.prod(L)) * nb
    op = lambda v: native.coarse_op_apply_herm_half(  # noqa: E731
        Ahalf, v.reshape(-1, nb, 1), L, pos_disp).reshape(-1)
    rec = dict(kappa_target=kappa, N=N, gen_seconds=round(tgen, 1))
    if N <= 8192:
        I = np.eye(N, dtype=np.complex128).reshape(-1, nb, N)
        Hd = native.coarse_op_apply_herm_half(Ahalf, I, L, pos_disp).reshape(N, N)
        ev = np.linalg.eigvalsh(0.5 * (Hd + np.conj(Hd.T)))
        lmin, lmax, bmin, bmax = float(ev[0]), float(ev[-1]), 0.0, 0.0
        rec["method"] = "dense eigvalsh"
    else:
        v0 = vectors(L, nb, 1, seed, stream=6).reshape(-1)
        lmin, lmax, bmin, bmax = lanczos_extremes(op, v0, steps)
        rec["method"] = f"lanczos {steps} steps (no reorthogonalisation)"
    c = (lmax - kappa * lmin) / (kappa - 1)
    rec.update(lambda_min_H0=lmin, lambda_max_H0=lmax, bound_min=bmin, bound_max=bmax,
               shift=c, lambda_min=lmin + c, lambda_max=lmax + c,
               gershgorin_radius_H0=gershgorin_radius(Ahalf),
               seconds=round(time.time() - t0, 1))
    op = None
    release_half(Ahalf)
    return rec


def main(argv=None):
    from synth import WORKLOADS
    ap = argparse.ArgumentParser()
    ap.add_argument("names", nargs="*")
    ap.add_argument("--steps", type=int, default=800)
    ap.add_argument("--procs", type=int, default=os.cpu_count() or 1)
    a = ap.parse_args(argv)
    names = a.names or list(WORKLOADS)
    table = {}
    if os.path.exists(OUT):
        with open(OUT) as f:
            table = json.load(f)
    for n in names:
        rec = estimate(WORKLOADS[n], a.steps, a.procs)
        rec["recipe"] = "c = (lam_max - kappa lam_min)/(kappa - 1) of the unshifted operator"
        table[n] = rec
        print(n, json.dumps(rec), flush=True)
        with open(OUT + ".tmp", "w") as f:
            json.dump(table, f, indent=1, sort_keys=True)
        os.replace(OUT + ".tmp", OUT)


if __name__ == "__main__":
    sys.exit(main())
