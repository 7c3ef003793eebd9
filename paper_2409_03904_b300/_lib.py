"""ctypes binding of libmrhs (include/mrhs.h): argument marshalling only.

Every computation runs in the CUDA library; this module checks tensor
dtypes/devices/contiguity, passes raw device pointers and the current torch
stream, and turns status codes into exceptions.  It raises at import-time
use if the shared library has not been built: there is no fallback.
"""
import ctypes
import os

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmrhs.so")

MRHS_OK = 0
ERRORS = {-1: "INVALID_ARG", -2: "CUDA", -3: "NOT_CONVERGED", -4: "BREAKDOWN", -5: "NONFINITE",
          -6: "UNSUPPORTED", -7: "NO_MEMORY", -8: "DEVICE"}
PREC = {"fp64": 0, "fp32": 1, "bf16": 2, "fp16": 3, "fp16x": 4, "tc32": 5, "df32": 6, "oz": 7}
NUM_PREC = 8
WIDE = ("fp64", "df32", "oz")    # precisions whose vectors are complex128
NAMES = {v: k for k, v in PREC.items()}
C128, C64 = 0, 1
MAX_RHS = 64
SOLVE_FP64, SOLVE_MIXED, SOLVE_CG5D = 0, 1, 2


class MrhsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class SolveParams(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("maxiter", ctypes.c_int32), ("mode", ctypes.c_int32),
                ("precond", ctypes.c_int32), ("precond_prec", ctypes.c_int32),
                ("cheb_order", ctypes.c_int32), ("cheb_lo", ctypes.c_double),
                ("cheb_hi", ctypes.c_double), ("inner_tol", ctypes.c_double),
                ("max_cycles", ctypes.c_int32), ("check_every", ctypes.c_int32),
                ("breakdown_tau", ctypes.c_double), ("krylov_prec", ctypes.c_int32),
                ("use_graph", ctypes.c_int32), ("residual_prec", ctypes.c_int32),
                ("recycle", ctypes.c_int32), ("recycle_max_blocks", ctypes.c_int32),
                ("fp64_prec", ctypes.c_int32), ("inner_tol_later", ctypes.c_double)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("iters", ctypes.c_int32), ("cycles", ctypes.c_int32),
                ("nrhs", ctypes.c_int32), ("applies", ctypes.c_int64 * NUM_PREC),
                ("resid", ctypes.c_double * MAX_RHS), ("cheb_lo", ctypes.c_double),
                ("cheb_hi", ctypes.c_double), ("ms_total", ctypes.c_double),
                ("krylov_prec", ctypes.c_int32), ("precond_prec", ctypes.c_int32),
                ("cycle_iters", ctypes.c_int32 * 16), ("cycle_resid", ctypes.c_double * 16),
                ("cycle_flag", ctypes.c_int32 * 16), ("recycle_blocks", ctypes.c_int32),
                ("recycle_projections", ctypes.c_int32)]

    def as_dict(self):
        return dict(status=self.status, iters=self.iters, cycles=self.cycles,
                    applies={k: int(self.applies[v]) for k, v in PREC.items()},
                    resid=[self.resid[j] for j in range(self.nrhs)], cheb_lo=self.cheb_lo,
                    cheb_hi=self.cheb_hi, ms_total=self.ms_total,
                    krylov_prec=NAMES.get(self.krylov_prec), precond_prec=NAMES.get(self.precond_prec),
                    cycle_iters=[self.cycle_iters[c] for c in range(min(self.cycles, 16))],
                    cycle_resid=[self.cycle_resid[c] for c in range(min(self.cycles, 16))],
                    cycle_flag=[self.cycle_flag[c] for c in range(min(self.cycles, 16))],
                    recycle_blocks=self.recycle_blocks,
                    recycle_projections=self.recycle_projections)


class TuneResult(ctypes.Structure):
    _fields_ = [("pts_per_stage", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("max_stages", ctypes.c_int32), ("candidates", ctypes.c_int32),
                ("ms", ctypes.c_double), ("ms_default", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None
P, I32, I64, D, U32 = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double,
                       ctypes.c_uint32)
SIGNATURES = {
    "mrhs_op_create": [ctypes.POINTER(P), P, I32, I32, P, P, U32, P],
    "mrhs_op_create_halo": [ctypes.POINTER(P), P, P, I32, I32, P, P, U32, P],
    "mrhs_gather_rows": [P, I64, P, I64, P, I64, P],
    "mrhs_col_dot": [P, P, P, I64, I32, I32, P],
    "mrhs_col_ratio": [P, P, P, P, I32, D, P],
    "mrhs_col_update": [P, P, P, D, I64, I32, I32, P],
    "mrhs_scatter_rows": [P, I64, P, P, I64, I64, P],
    "mrhs_op_destroy": [P],
    "coarse_op_apply": [P, I32, P, P, I32, P],
    "coarse_op_apply_dag": [P, I32, P, P, I32, P],
    "block_inner": [P, P, P, I64, I32, I32, I32, P],
    "coarse_op_outer": [P, P, P, P, D, I32, I32, P],
    "block_inner_noalloc": [P, P, P, I64, I32, I32, I32, P],
    "block_axpy": [P, P, P, D, I64, I32, I32, I32, P],
    "herm_factor": [P, P, P, P, I32, D, P],  # rank: device int32*
    "cheby_apply": [P, I32, D, D, I32, P, P, I32, P],
    "coarse_solve_defl_cheby": [P, I32, P, P, I32, D, D, I32, P, P, I32, P],
    "block_project": [P, P, P, I64, I32, I32, I32, I32, P],
    "coarsen_op": [P, P, P, I32, P, I32, P, P],
    "block_promote": [P, P, P, I64, I32, I32, I32, I32, P],
    "block_cg_solve": [P, P, P, I32, ctypes.POINTER(SolveParams), ctypes.POINTER(SolveInfo), P],
    "mrhs_solve_params_default": [ctypes.POINTER(SolveParams), I32],
    "mrhs_last_error": [],
    "mrhs_version": [],
    "mrhs_device_error": [],
    "mrhs_debug_wait_limit": [ctypes.c_uint64],
    "mrhs_block_tc": [I32],
    "mrhs_op_kernel_timing": [P, I32],
    "mrhs_op_kernel_time": [P, I32, P, P],
    "mrhs_launch_count": [],
    "mrhs_op_lambda_max": [P, I32, I32, P, P],
    "mrhs_op_tc_tune": [P, I32, I32, I32],
    "mrhs_op_hermitian": [P, I32, P],
    "mrhs_batch_apply": [P, I32, I32, P, P, P, P],
    "mrhs_batch_solve": [P, I32, P, P, P, ctypes.POINTER(SolveParams), P, P],
    "mrhs_autotune": [P, I32, I32, P, I32, ctypes.POINTER(TuneResult), P],
    "mrhs_autotune_save": [ctypes.c_char_p],
    "mrhs_autotune_load": [ctypes.c_char_p],
    "mrhs_autotune_entries": [],
    "mrhs_autotune_clear": [],
}


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with "
                              "`python -m paper_2409_03904_b300.build` (no CPU fallback exists)")
        l = ctypes.CDLL(LIB_PATH)
        for name, args in SIGNATURES.items():
            f = getattr(l, name)
            f.argtypes = args
            f.restype = ctypes.c_int32
        l.mrhs_last_error.restype = ctypes.c_char_p
        l.mrhs_version.restype = ctypes.c_char_p
        l.mrhs_solve_params_default.restype = None
        l.mrhs_launch_count.restype = ctypes.c_int64
        l.mrhs_autotune_entries.restype = ctypes.c_int64
        l.mrhs_autotune_clear.restype = None
        _lib = l
    return _lib


def check(code):
    if code != MRHS_OK:
        raise MrhsError(code, lib().mrhs_last_error().decode())


def stream_ptr(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def dev_ptr(t, dtype=None, name="tensor"):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def vec_dtype(prec):
    return torch.complex128 if prec in WIDE else torch.complex64
