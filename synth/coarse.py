"""Seeded synthetic coarse operators and multi-RHS sources.

The paper's operators come from gauge ensembles that are not available, so
every workload is synthetic.  The recipe (no solver arithmetic here, only
random draws and index bookkeeping):

* lattice L = (L0, L1, L2, L3), periodic, site x = x0 + L0*(x1 + L1*(x2 + L2*x3));
* stencil: displacement list delta_p, p = 0 the self term (9-point: self and
  +-e_mu; 81-point: all of {-1,0,1}^4, the full neighbourhood of Sec. 2.6
  "Coarse operator");
* hop matrices: A_p(x) = G / sqrt(nb) with G i.i.d. standard complex normal
  for every "positive" delta_p (first non-zero component +1); the partner is
  fixed by Hermiticity of the operator, A_{-p}(x + delta_p) = A_p(x)^dagger;
* self term: A_0(x) = (G + G^dagger)/2 / sqrt(nb) + c I, with the shift c read
  from a table that the oracle's Lanczos script writes so that the condition
  number hits its target;
* sources and other vectors: standard complex normal, layout [V][nb][nrhs].

Counter layout of each Philox draw: (c0, c1, c2, c3) = (element, site,
stencil point or row, stream).
"""
import itertools
import json
import os

import numpy as np

from .philox import complex_normal

BASE_SEED = 2409039040
STREAM_HOP = 1
STREAM_SELF = 2
STREAM_B = 3
STREAM_W = 4
STREAM_X0 = 5
STREAM_U = 6

_SHIFT_TABLE = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                            "tests", "golden", "shifts.json")


def stencil(npts):
    """Return (disp int8 [npts][4], pair int32 [npts]) with p = 0 the self term.

    pair[p] is the index of -delta_p.
    """
    if npts == 9:
        d = [(0, 0, 0, 0)]
        for mu in range(4):
            for s in (1, -1):
                e = [0, 0, 0, 0]
                e[mu] = s
                d.append(tuple(e))
    elif npts == 81:
        d = [(0, 0, 0, 0)]
        for t in itertools.product((-1, 0, 1), repeat=4):
            if t != (0, 0, 0, 0):
                d.append(t)
    elif npts == 1:
        d = [(0, 0, 0, 0)]
    else:
        raise ValueError("stencil size must be 1, 9 or 81")
    disp = np.array(d, dtype=np.int8)
    index = {tuple(int(v) for v in row): i for i, row in enumerate(disp)}
    pair = np.array([index[tuple(-int(v) for v in row)] for row in disp], dtype=np.int32)
    return disp, pair


def is_positive(delta):
    for v in delta:
        if v != 0:
            return v > 0
    return False


def volume(L):
    return int(np.prod(L))


def site_coords(L, sites):
    sites = np.asarray(sites, dtype=np.int64)
    x0 = sites % L[0]
    r = sites // L[0]
    x1 = r % L[1]
    r = r // L[1]
    x2 = r % L[2]
    x3 = r // L[2]
    return np.stack([x0, x1, x2, x3], axis=-1)


def site_index(L, coords):
    c = np.asarray(coords, dtype=np.int64)
    return c[..., 0] + L[0] * (c[..., 1] + L[1] * (c[..., 2] + L[2] * c[..., 3]))


def shifted_sites(L, sites, delta):
    """Periodic x + delta for an array of site indices."""
    c = site_coords(L, sites) + np.asarray(delta, dtype=np.int64)
    c = np.mod(c, np.asarray(L, dtype=np.int64))
    return site_index(L, c)


def _gauss_block(nb, sites, p, stream, seed):
    """[len(sites)][nb][nb] standard complex normals for (site, p, stream)."""
    e = np.arange(nb * nb, dtype=np.int64).reshape(1, nb, nb)
    s = np.asarray(sites, dtype=np.int64).reshape(-1, 1, 1)
    return complex_normal(e, s, p, stream, seed)


def coarse_op(L, nb, npts, seed, shift, sites=None, points=None):
    """Canonical coefficients A[x][p][a][b] (complex128) for the given sites.

    sites defaults to the whole lattice; points defaults to all stencil points
    (then the result is [len(sites)][npts][nb][nb]).
    """
    disp, pair = stencil(npts)
    if sites is None:
        sites = np.arange(volume(L), dtype=np.int64)
    sites = np.asarray(sites, dtype=np.int64)
    if points is None:
        points = range(npts)
    points = list(points)
    out = np.empty((len(sites), len(points), nb, nb), dtype=np.complex128)
    inv = 1.0 / np.sqrt(nb)
    for k, p in enumerate(points):
        d = tuple(int(v) for v in disp[p])
        if d == (0, 0, 0, 0):
            g = _gauss_block(nb, sites, 0, STREAM_SELF, seed) * inv
            blk = 0.5 * (g + np.conj(np.swapaxes(g, -1, -2)))
            blk = blk + shift * np.eye(nb)[None]
        elif is_positive(d):
            blk = _gauss_block(nb, sites, p, STREAM_HOP, seed) * inv
        else:
            q = int(pair[p])
            src = shifted_sites(L, sites, d)           # x + delta_p, where A_q was drawn
            g = _gauss_block(nb, src, q, STREAM_HOP, seed) * inv
            blk = np.conj(np.swapaxes(g, -1, -2))
        out[:, k] = blk
    return out


def vectors(L, nb, nrhs, seed, stream=STREAM_B, sites=None):
    """[len(sites)][nb][nrhs] standard complex normals (column r is RHS r)."""
    if sites is None:
        sites = np.arange(volume(L), dtype=np.int64)
    s = np.asarray(sites, dtype=np.int64).reshape(-1, 1, 1)
    a = np.arange(nb, dtype=np.int64).reshape(1, nb, 1)
    r = np.arange(nrhs, dtype=np.int64).reshape(1, 1, nrhs)
    return complex_normal(r, s, a, stream, seed)


def load_shift(name):
    """Shift c of the self term for a named workload (written by the oracle's
    Lanczos script into tests/golden/shifts.json)."""
    with open(_SHIFT_TABLE) as f:
        table = json.load(f)
    if name not in table:
        raise KeyError(f"no shift recorded for workload {name!r}")
    return float(table[name]["shift"])
