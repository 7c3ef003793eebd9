"""Seeded input generators: Philox known answers, distribution, Hermitian
pairing of the hop matrices, stencil geometry."""
import os

import numpy as np

from synth import coarse_op, complex_normal, philox4x32_10, stencil, vectors
from synth.coarse import is_positive, shifted_sites

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answers():
    rows = []
    with open(os.path.join(GOLDEN, "philox_kat.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([int(w, 16) for w in line.split()])
    assert len(rows) == 3
    for r in rows:
        out = philox4x32_10(r[0], r[1], r[2], r[3], r[4], r[5])
        assert [int(v) for v in out] == r[6:]


def test_philox_vectorised_matches_scalar():
    c0 = np.arange(17)
    out = philox4x32_10(c0, 5, 7, 9, 123, 456)
    for i in (0, 3, 16):
        one = philox4x32_10(i, 5, 7, 9, 123, 456)
        assert all(int(a[i]) == int(b) for a, b in zip(out, one))


def test_complex_normal_moments():
    z = complex_normal(np.arange(200000), 1, 2, 3, 99)
    assert abs(np.mean(np.abs(z) ** 2) - 1.0) < 0.01
    assert abs(np.mean(z.real)) < 0.01 and abs(np.mean(z.imag)) < 0.01
    assert abs(np.var(z.real) - 0.5) < 0.01
    assert abs(np.mean(z.real * z.imag)) < 0.01


def test_stencils():
    for n in (9, 81):
        d, pair = stencil(n)
        assert d.shape == (n, 4) and tuple(d[0]) == (0, 0, 0, 0)
        assert len({tuple(r) for r in d}) == n
        for p in range(n):
            assert np.array_equal(d[pair[p]], -d[p])
        npos = sum(is_positive(tuple(r)) for r in d)
        assert npos == (n - 1) // 2


def test_hermitian_pairing():
    L = (3, 2, 3, 2)
    for npts in (9, 81):
        A = coarse_op(L, 3, npts, 777, 0.5)
        d, pair = stencil(npts)
        V = int(np.prod(L))
        for p in range(npts):
            y = shifted_sites(L, np.arange(V), d[p])
            # A_{-p}(x + delta_p) = A_p(x)^dagger
            lhs = A[y, pair[p]]
            rhs = np.conj(np.swapaxes(A[:, p], -1, -2))
            assert np.array_equal(lhs, rhs)


def test_site_subset_consistent():
    L = (4, 3, 2, 3)
    A = coarse_op(L, 4, 81, 31, 1.0)
    sites = np.array([0, 5, 17, 71])
    As = coarse_op(L, 4, 81, 31, 1.0, sites=sites)
    assert np.array_equal(A[sites], As)
    B = vectors(L, 4, 6, 31)
    Bs = vectors(L, 4, 3, 31, sites=sites)
    assert np.array_equal(B[sites][:, :, :3], Bs)


def test_covariant_laplacian():
    """Links unitary; the operator Hermitian with its spectrum in [m, 16 + m];
    at eps = 0 it is the free Laplacian, whose eigenvalues are
    8 + m - 2 sum_mu cos(2 pi k_mu / L_mu), each nb times."""
    import numpy as np
    from synth.laplace import covariant_laplacian, links
    from tests.test_oracle_ops import dense_matrix
    from synth import stencil
    L, nb, m = (3, 2, 2, 3), 3, 0.25
    U = links(L, nb, 0.4, 11)
    assert np.allclose(np.conj(np.swapaxes(U, -1, -2)) @ U, np.eye(nb), atol=1e-13)
    disp, _ = stencil(9)
    H = dense_matrix(covariant_laplacian(L, nb, 0.4, m, 11), L, disp)
    assert np.allclose(H, np.conj(H.T), atol=1e-13)
    ev = np.linalg.eigvalsh(H)
    assert ev[0] >= m - 1e-12 and ev[-1] <= 16 + m + 1e-12
    H0 = dense_matrix(covariant_laplacian(L, nb, 0.0, m, 11), L, disp)
    k = np.meshgrid(*[np.arange(l) for l in L], indexing="ij")
    lam = 8 + m - 2 * sum(np.cos(2 * np.pi * k[mu] / L[mu]) for mu in range(4))
    ref = np.sort(np.repeat(lam.reshape(-1), nb))
    assert np.allclose(np.linalg.eigvalsh(H0), ref, atol=1e-12)
