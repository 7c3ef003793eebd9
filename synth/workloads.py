"""Named synthetic workloads (lattice, basis size, stencil, RHS count, target
condition number, tolerance, seed).  Sizes follow the coarse problems the
paper solves: 4^4 coarse blocks of a fine lattice, n_basis 16..64, 9- or
81-point stencils and about a dozen right-hand sides (Sec. 2.6, Table 1,
Table 6).  Seeds are BASE_SEED + index.
"""
from .coarse import BASE_SEED

_LIST = [
    # name, L, nb, npts, nrhs, kappa, tol
    ("L4_nb24_9pt_r4", (4, 4, 4, 4), 24, 9, 4, 1e3, 1e-10),
    ("L8_nb32_81pt_r16", (8, 8, 8, 8), 32, 81, 16, 1e4, 1e-8),
    ("L6_nb16_9pt_r8", (6, 6, 6, 6), 16, 9, 8, 1e3, 1e-10),
    ("L12_nb48_81pt_r32", (12, 12, 12, 12), 48, 81, 32, 1e4, 1e-8),
]

# twelve independent problems solved side by side in one batched launch
_BATCH = [
    ((4, 4, 4, 4), 24, 4, 9, 1e3),
    ((4, 4, 4, 4), 32, 8, 81, 1e4),
    ((4, 4, 4, 4), 48, 16, 9, 3e3),
    ((6, 6, 6, 6), 24, 12, 81, 1e3),
    ((6, 6, 6, 6), 32, 24, 9, 1e4),
    ((6, 6, 6, 6), 48, 4, 81, 3e3),
    ((8, 8, 8, 8), 24, 16, 9, 1e4),
    ((8, 8, 8, 8), 32, 4, 81, 3e3),
    ((8, 8, 8, 8), 48, 8, 9, 1e3),
    ((6, 6, 6, 6), 32, 16, 81, 1e3),
    ((4, 4, 4, 4), 24, 24, 81, 1e4),
    ((8, 8, 8, 8), 48, 12, 81, 1e4),
]


def _mk(name, L, nb, npts, nrhs, kappa, tol, seed):
    return dict(name=name, L=tuple(L), nb=nb, npts=npts, nrhs=nrhs, kappa=kappa,
                tol=tol, seed=seed)


WORKLOADS = {}
for _i, (_n, _L, _nb, _np, _r, _k, _t) in enumerate(_LIST):
    WORKLOADS[_n] = _mk(_n, _L, _nb, _np, _r, _k, _t, BASE_SEED + (_i if _i < 3 else 4))

BATCH = []
for _j, (_L, _nb, _r, _np, _k) in enumerate(_BATCH):
    _n = f"batch{_j:02d}_L{_L[0]}_nb{_nb}_{_np}pt_r{_r}"
    BATCH.append(_mk(_n, _L, _nb, _np, _r, _k, 1e-8, BASE_SEED + 3 + 1000 * (_j + 1)))
    WORKLOADS[_n] = BATCH[-1]
