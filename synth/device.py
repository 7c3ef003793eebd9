"""Device-side generation of the same seeded inputs (synth/csrc/synth_gen.cu),
for lattices whose coefficients are too large to draw on the host.  Random
draws and index bookkeeping only; values agree with synth.coarse to the last
few ulps (the CUDA and numpy log/cos/sin may round differently).
"""
import ctypes
import os
import subprocess

import numpy as np
import torch

from .coarse import STREAM_B, stencil, volume

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "csrc", "synth_gen.cu")
_OUT = os.path.join(_HERE, "_build", "libsynth_gen.so")
_lib = None


def build(force=False):
    if not force and os.path.exists(_OUT) and os.path.getmtime(_OUT) >= os.path.getmtime(_SRC):
        return _OUT
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    nvcc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    tmp = _OUT + f".{os.getpid()}.tmp"
    subprocess.check_call([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3",
                           "-Xcompiler", "-fPIC", "-shared", "-o", tmp, _SRC])
    os.replace(tmp, _OUT)
    return _OUT


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P, I32, I64, U32, U64, D = (ctypes.c_void_p, ctypes.c_int, ctypes.c_int64,
                                    ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double)
        _lib.synth_gen_op.argtypes = [P, I64, I32, I32, P, P, P, U64, D, P]
        _lib.synth_gen_vec.argtypes = [P, I64, I32, I32, U64, U32, P]
        _lib.synth_philox_words.argtypes = [P, I64, U32, U32, U32, U64, P]
    return _lib


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def coarse_op(L, nb, npts, seed, shift, device="cuda"):
    """Device tensor [V][npts][nb][nb] complex128, same recipe as synth.coarse_op."""
    lib = _load()
    disp, pair = stencil(npts)
    V = volume(L)
    A = torch.empty((V, npts, nb, nb), dtype=torch.complex128, device=device)
    d_disp = torch.from_numpy(np.ascontiguousarray(disp)).to(device)
    d_pair = torch.from_numpy(pair.astype(np.int32)).to(device)
    Lc = (ctypes.c_int32 * 4)(*[int(v) for v in L])
    rc = lib.synth_gen_op(ctypes.c_void_p(A.data_ptr()), V, nb, npts, Lc,
                          ctypes.c_void_p(d_disp.data_ptr()), ctypes.c_void_p(d_pair.data_ptr()),
                          seed, float(shift), _stream())
    if rc:
        raise RuntimeError(f"synth_gen_op: cuda error {rc}")
    torch.cuda.current_stream().synchronize()
    return A


def vectors(L, nb, nrhs, seed, stream=STREAM_B, device="cuda"):
    lib = _load()
    V = volume(L)
    X = torch.empty((V, nb, nrhs), dtype=torch.complex128, device=device)
    rc = lib.synth_gen_vec(ctypes.c_void_p(X.data_ptr()), V, nb, nrhs, seed, stream, _stream())
    if rc:
        raise RuntimeError(f"synth_gen_vec: cuda error {rc}")
    return X


def philox_words(n, c1, c2, c3, seed, device="cuda"):
    """[n][4] uint32 words for counters (i, c1, c2, c3), i < n (as int64 tensor)."""
    lib = _load()
    out = torch.empty((n, 4), dtype=torch.int32, device=device)
    rc = lib.synth_philox_words(ctypes.c_void_p(out.data_ptr()), n, c1, c2, c3, seed, _stream())
    if rc:
        raise RuntimeError(f"synth_philox_words: cuda error {rc}")
    return out.to(torch.int64) & 0xFFFFFFFF
