"""Build libmrhs.so (CUDA, sm_103a) in-tree with nvcc.

    python -m paper_2409_03904_b300.build [--force] [-j N]

Every .cu under csrc/ is compiled separately (-gencode arch=compute_103a,
code=sm_103a, -O3 -lineinfo) into _build/ and linked into one shared object
next to this file.  Only sources newer than their object are recompiled.
"""
import argparse
import concurrent.futures as cf
import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")
NVCC = os.path.join(CUDA, "bin", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-I", os.path.join(ROOT, "include"), "-I", os.path.join(HERE, "csrc")]
LIB = os.path.join(HERE, "libmrhs.so")


def _objects(src_dir, build_dir):
    srcs = sorted(glob.glob(os.path.join(src_dir, "*.cu")))
    return [(s, os.path.join(build_dir, os.path.basename(s)[:-3] + ".o")) for s in srcs]


def _stale(obj, deps):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


def build_library(src_dir, build_dir, out, extra=(), force=False, jobs=8, verbose=False):
    os.makedirs(build_dir, exist_ok=True)
    headers = glob.glob(os.path.join(src_dir, "*.cuh")) + glob.glob(os.path.join(ROOT, "include", "*.h"))
    pairs = _objects(src_dir, build_dir)
    todo = [(s, o) for s, o in pairs if force or _stale(o, [s] + headers)]

    def one(so):
        s, o = so
        cmd = [NVCC] + ARCH + FLAGS + list(extra) + ["-c", s, "-o", o]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        return s, r.returncode, r.stdout + r.stderr

    failed = []
    with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
        for s, rc, log in ex.map(one, todo):
            if log.strip() and (rc or verbose):
                sys.stderr.write(log)
            if rc:
                failed.append(s)
    if failed:
        raise RuntimeError("nvcc failed for: " + ", ".join(failed))
    objs = [o for _, o in pairs]
    if force or todo or _stale(out, objs):
        tmp = out + f".{os.getpid()}.tmp"
        cmd = [NVCC] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"]
        subprocess.check_call(cmd)
        os.replace(tmp, out)
    return out


def build(force=False, jobs=8, verbose=False):
    return build_library(os.path.join(HERE, "csrc"), os.path.join(HERE, "_build"), LIB,
                         force=force, jobs=jobs, verbose=verbose)


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--force", action="store_true")
    ap.add_argument("-j", type=int, default=8)
    ap.add_argument("-v", action="store_true", help="print ptxas resource usage")
    a = ap.parse_args()
    print(build(force=a.force, jobs=a.j, verbose=a.v))
