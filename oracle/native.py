"""ctypes binding of the C oracle operator (oracle/csrc/oracle_op.c).

Test infrastructure only (see the package docstring).  The shared object is
compiled with gcc on first use (or by the package build step) into
oracle/_build/.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "csrc", "oracle_op.c")
_OUT = os.path.join(_HERE, "_build", "liboracle_op.so")
_lib = None


def build(force=False):
    """Compile the C oracle with gcc -O2 -fopenmp (no fast-math: IEEE FP64)."""
    if not force and os.path.exists(_OUT) and os.path.getmtime(_OUT) >= os.path.getmtime(_SRC):
        return _OUT
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    tmp = _OUT + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                           "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _OUT)
    return _OUT


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i32, i64 = ctypes.c_int32, ctypes.c_int64
        _lib.oracle_op_apply.argtypes = [P, P, P, P, i32, i32, P, i32]
        _lib.oracle_op_apply_sites.argtypes = [P, P, P, P, i32, i32, P, i32, P, i64]
        _lib.oracle_op_apply_herm_half.argtypes = [P, P, P, P, i32, i32, P, i32]
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def coarse_op_apply(A, X, L, disp):
    """Same definition as oracle.ops.coarse_op_apply, in C."""
    lib = _load()
    A = np.ascontiguousarray(A, dtype=np.complex128)
    X = np.ascontiguousarray(X, dtype=np.complex128)
    Lc = np.asarray(L, dtype=np.int32)
    d = np.ascontiguousarray(disp, dtype=np.int8)
    Y = np.empty_like(X)
    lib.oracle_op_apply(_ptr(A), _ptr(X), _ptr(Y), _ptr(Lc), A.shape[2], A.shape[1], _ptr(d),
                        X.shape[2])
    return Y


def coarse_op_apply_sites(A_sites, X, L, disp, sites):
    """Rows Y(s) for the listed sites only; A_sites[s] holds those sites'
    coefficients, X is the full input vector."""
    lib = _load()
    A_sites = np.ascontiguousarray(A_sites, dtype=np.complex128)
    X = np.ascontiguousarray(X, dtype=np.complex128)
    Lc = np.asarray(L, dtype=np.int32)
    d = np.ascontiguousarray(disp, dtype=np.int8)
    s = np.ascontiguousarray(sites, dtype=np.int64)
    Y = np.empty((len(s), X.shape[1], X.shape[2]), dtype=np.complex128)
    lib.oracle_op_apply_sites(_ptr(A_sites), _ptr(X), _ptr(Y), _ptr(Lc), A_sites.shape[2],
                              A_sites.shape[1], _ptr(d), X.shape[2], _ptr(s), len(s))
    return Y


def coarse_op_apply_herm_half(Ahalf, X, L, pos_disp):
    """Hermitian stencil from its self and positive-displacement blocks."""
    lib = _load()
    Ahalf = np.ascontiguousarray(Ahalf, dtype=np.complex128)
    X = np.ascontiguousarray(X, dtype=np.complex128)
    Lc = np.asarray(L, dtype=np.int32)
    d = np.ascontiguousarray(pos_disp, dtype=np.int8).reshape(-1, 4)
    Y = np.empty_like(X)
    lib.oracle_op_apply_herm_half(_ptr(Ahalf), _ptr(X), _ptr(Y), _ptr(Lc), Ahalf.shape[2],
                                  d.shape[0], _ptr(d), X.shape[2])
    return Y
