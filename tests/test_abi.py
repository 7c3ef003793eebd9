"""The C ABI library builds for sm_103a, loads on a machine without a GPU and
exports every function that include/*.h declares (no compute calls here)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?\w+\s*\*?\s*(\w+)\s*\(", src, flags=re.M):
            if m.group(1) not in ("if", "return", "sizeof"):
                names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def libpath():
    from paper_2409_03904_b300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("mrhs_op_create", "mrhs_op_destroy", "coarse_op_apply", "coarse_op_apply_dag",
              "block_inner", "block_axpy", "herm_factor", "cheby_apply", "block_cg_solve",
              "mrhs_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_errors_without_gpu_are_codes_not_crashes(libpath):
    import paper_2409_03904_b300 as mrhs
    l = mrhs._lib.lib()
    assert b"sm_103a" in l.mrhs_version()
    # null arguments are rejected before any CUDA call
    rc = l.block_inner(None, None, None, 10, 2, 2, 0, None)
    assert rc == -1 and b"null" in l.mrhs_last_error()
    rc = l.block_axpy(None, None, None, 0.0, -1, 2, 2, 0, None)
    assert rc == -1


def test_no_oracle_in_product_path():
    """The package and its CUDA sources never reference the oracle."""
    for f in glob.glob(os.path.join(ROOT, "paper_2409_03904_b300", "**", "*"), recursive=True):
        if os.path.isfile(f) and f.endswith((".py", ".cu", ".cuh", ".h")):
            assert "oracle" not in open(f).read().lower(), f


def test_ctypes_structs_match_the_header(tmp_path):
    """The Python mirrors of mrhs_solve_params / mrhs_solve_info / mrhs_tune_result
    have the C layout: sizes and field offsets from a C program built against
    include/mrhs.h with the host compiler."""
    from paper_2409_03904_b300 import _lib
    structs = {"mrhs_solve_params": _lib.SolveParams, "mrhs_solve_info": _lib.SolveInfo,
               "mrhs_tune_result": _lib.TuneResult}
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "mrhs.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'  printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    import subprocess
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    got = {}
    for line in out.splitlines():
        name, field, val = line.split()
        got[(name, field)] = int(val)
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)


def test_solve_parameter_defaults(libpath):
    """mrhs_solve_params_default is host code, checked here without a GPU:
    the defaults per mode, including the mixed solve's later-cycle inner
    target (1e-2, 0 elsewhere) and the automatic precision choices (-1)."""
    import paper_2409_03904_b300 as mrhs
    l = mrhs._lib.lib()
    want_common = dict(tol=1e-8, maxiter=5000, precond_prec=-1, krylov_prec=-1, use_graph=1,
                       residual_prec=-1, cheb_order=8, cheb_lo=0.0, cheb_hi=0.0, inner_tol=1e-3,
                       max_cycles=12, check_every=4, breakdown_tau=1e-12, recycle=0,
                       recycle_max_blocks=0, fp64_prec=-1)
    for mode, precond, later in ((mrhs.SOLVE_FP64, 0, 0.0), (mrhs.SOLVE_MIXED, 1, 1e-2),
                                 (mrhs.SOLVE_CG5D, 0, 0.0)):
        p = mrhs._lib.SolveParams()
        l.mrhs_solve_params_default(ctypes.byref(p), mode)
        got = {k: getattr(p, k) for k in want_common}
        assert got == want_common, (mode, got)
        assert (p.mode, p.precond, p.inner_tol_later) == (mode, precond, later)
    l.mrhs_solve_params_default(None, mrhs.SOLVE_MIXED)      # a null pointer is ignored
