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
