"""block_inner_noalloc: the Gram product for callers that may not allocate.

Callers whose device memory belongs to someone else's pool, or who may not
let a cudaMalloc (and the device synchronisation it can bring) happen inside
their loop, use this variant: its partial sums live in a fixed array inside
the library instead of a workspace the library allocates.  This file checks,
through the C ABI, that two calls in a row give the same Gram as the
allocating entry point block_inner, within the tolerance of the other Gram
tests.  It is collected last so that a run stopping at the first failure has
already run everything else; it also passes when run on its own.
"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _noalloc(lib, X, Y, G, N, rx, ry, dtype):
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.block_inner_noalloc(ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(Y.data_ptr()),
                                   ctypes.c_void_p(G.data_ptr()), N, rx, ry, dtype, s)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_noalloc_gram_matches_block_inner_twice(dtype):
    assert torch.cuda.is_available()
    import paper_2409_03904_b300 as mrhs
    lib = mrhs._lib.lib()
    tdt = torch.complex128 if dtype == "c128" else torch.complex64
    code = mrhs.C128 if dtype == "c128" else mrhs.C64
    tol = 1e-13 if dtype == "c128" else 1e-6
    rng = np.random.default_rng(2024)
    # two calls in a row with different shapes: the second reuses the array
    for N, rx, ry in ((200003, 32, 32), (70001, 64, 12)):
        X = torch.from_numpy(rng.standard_normal((N, rx)) + 1j * rng.standard_normal((N, rx)))
        Y = torch.from_numpy(rng.standard_normal((N, ry)) + 1j * rng.standard_normal((N, ry)))
        X, Y = X.to(tdt).cuda(), Y.to(tdt).cuda()
        G = torch.full((rx, ry), float("nan"), dtype=torch.complex128, device="cuda")
        assert _noalloc(lib, X, Y, G, N, rx, ry, code) == 0, lib.mrhs_last_error()
        ref = mrhs.block_inner(X, Y)
        torch.cuda.synchronize()
        scale = float(torch.linalg.norm(X.to(torch.complex128)) * torch.linalg.norm(Y.to(torch.complex128)))
        assert float(torch.linalg.norm(G - ref)) <= tol * scale
        G2 = torch.empty_like(G)
        assert _noalloc(lib, X, Y, G2, N, rx, ry, code) == 0
        torch.cuda.synchronize()
        assert torch.equal(G, G2)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import paper_2409_03904_b300 as mrhs
    lib = mrhs._lib.lib()
    X = torch.zeros((16, 65), dtype=torch.complex128, device="cuda")
    G = torch.zeros((65, 65), dtype=torch.complex128, device="cuda")
    assert _noalloc(lib, X, X, G, 16, 65, 65, mrhs.C128) == -1
    assert b"64" in lib.mrhs_last_error()


def test_noalloc_takes_no_device_memory_after_set_up():
    """After one set-up call (which loads the library's device code and so
    its static array), calls with shapes that would make block_inner grow its
    workspace leave the device's free memory unchanged."""
    import paper_2409_03904_b300 as mrhs
    lib = mrhs._lib.lib()
    shapes = ((4096, 8, 8), (1000003, 64, 64), (300001, 48, 17))
    rng = np.random.default_rng(77)
    bufs = []
    for N, rx, ry in shapes:
        X = torch.from_numpy(rng.standard_normal((N, rx)) + 1j * rng.standard_normal((N, rx))).cuda()
        Y = torch.from_numpy(rng.standard_normal((N, ry)) + 1j * rng.standard_normal((N, ry))).cuda()
        G = torch.empty((rx, ry), dtype=torch.complex128, device="cuda")
        bufs.append((X, Y, G, N, rx, ry))
    Z = torch.zeros((1, 1), dtype=torch.complex128, device="cuda")
    assert _noalloc(lib, Z, Z, Z, 0, 1, 1, mrhs.C128) == 0      # set-up call
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for X, Y, G, N, rx, ry in bufs:
        assert _noalloc(lib, X, Y, G, N, rx, ry, mrhs.C128) == 0, lib.mrhs_last_error()
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    X, Y, G, N, rx, ry = bufs[1]
    ref = X.conj().T @ Y
    assert float(torch.linalg.norm(G - ref)) <= 1e-13 * float(torch.linalg.norm(X) * torch.linalg.norm(Y))
