#!/usr/bin/env python
"""Benchmark: block-CG time to a 1e-8 residual per right-hand side (mixed
precision vs plain FP64) and the coarse operator's TFLOP/s at 32 RHS.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload NAME] [--op PREC [--lattice a,b,c,d]]

Workload (default): 12^4 coarse lattice, nb = 48, 81-point stencil, 32
right-hand sides, condition ~1e4, synthetic seeded operator and sources
(see synth/).  One step = one complete mixed-precision solve to a true FP64
relative residual of 1e-8 on every RHS: FP64 outer defect correction (true
residual, solution update), complex64 inner block CG with the TC32
tensor-core operator and a degree-8 Chebyshev preconditioner applied with the
FP16X tensor-core operator, each refinement cycle after the first started
from the Galerkin correction over the earlier cycles' search blocks (one
sweep, --recycle).  value = ms per RHS (lower is better).

--op PREC: one step = one application of the coarse operator in precision
PREC at the workload's shape (optionally on another lattice, same per-site
work); value = TFLOP/s (8 nb^2 nrhs npts V flop per application).

Multi-GPU (torchrun): the solve does not shard in this build; every rank
solves its own independent batch of right-hand sides against its own copy of
the operator (replicas, weak scaling), value = max time / all RHS.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WIDE = ("fp64", "df32", "oz")      # precisions whose vectors are complex128
METRIC = ("coarse-op TFLOP/s at Nrhs=32; block-CG time-to-1e-8 per RHS, mixed vs FP64")
DEFAULT_WORKLOAD = "L12_nb48_81pt_r32"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--precond", default="fp16x", choices=["fp16x", "fp16", "bf16", "fp32", "tc32"])
    ap.add_argument("--krylov", default="tc32", choices=["tc32", "fp32"])
    ap.add_argument("--residual", default="oz", choices=["oz", "df32", "fp64"],
                    help="operator of the refinement cycles' residuals (the one that meets "
                         "tol is always recomputed with the FP64 operator)")
    ap.add_argument("--fp64-op", default="oz", choices=["oz", "fp64"],
                    help="the FP64 operator: of the residual that decides convergence and of "
                         "the plain FP64 block CG (oz: digit-sliced tensor-core form held to the "
                         "FP64 tolerance; fp64: the FP64 pipes)")
    ap.add_argument("--cheb-order", type=int, default=8)
    ap.add_argument("--cheb-ratio", type=float, default=400.0, help="hi / lo")
    ap.add_argument("--inner-tol", type=float, default=3e-4,
                    help="inner block-CG target of the first refinement cycle (3e-4: 24 "
                         "iterations at 12^4; 1e-4 the same, 1e-3 20 but 4 more in the later "
                         "cycles)")
    ap.add_argument("--inner-tol-later", type=float, default=1e-2,
                    help="inner target of the later refinement cycles, which the Krylov "
                         "operator's own error limits to 1.5-2%% of their start at 12^4 "
                         "(1e-2 .. 4e-2: 42 inner iterations on four right-hand-side sets, "
                         "against 50-54 for 3e-4; 0: --inner-tol)")
    ap.add_argument("--recycle", type=int, default=1,
                    help="sweeps of the Galerkin start over the earlier cycles' search blocks "
                         "(0: plain restart; 1, the default: 60 instead of 66 inner "
                         "iterations at 12^4, a net gain with the tensor-core block algebra)")
    ap.add_argument("--rhs-offset", type=int, default=0,
                    help="solve: draw the right-hand sides from the workload's seed plus this offset")
    ap.add_argument("--check-every", type=int, default=4,
                    help="block-CG iterations between convergence checks (one graph chunk); "
                         "4: 42 inner iterations on each of four right-hand-side sets at 12^4 "
                         "with one recycling sweep and the later-cycle target, against 44 for "
                         "2 and 47 for 3")
    ap.add_argument("--fp64-native-iters", type=int, default=3,
                    help="iterations of plain FP64 block CG on the FP64 pipes timed for the "
                         "per-iteration comparison (0: skip)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the standalone operator, FP64 and e2e measurements")
    ap.add_argument("--cpu-sites", type=int, default=96, help="oracle sample size (sites)")
    ap.add_argument("--op", default=None,
                    choices=["fp64", "df32", "oz", "fp32", "bf16", "fp16", "fp16x", "tc32"],
                    help="time the coarse operator alone in this precision")
    ap.add_argument("--lattice", default=None, help="a,b,c,d: override the workload's lattice "
                    "(same per-site work; for profiling captures on a smaller case)")
    ap.add_argument("--nrhs", type=int, default=None, help="operator mode: right-hand sides")
    ap.add_argument("--nrhs-list", default=None, metavar="R1,R2,...",
                    help="operator mode: one operator, one JSON line per number of right-hand sides")
    ap.add_argument("--nb", type=int, default=None, help="operator mode: basis size")
    ap.add_argument("--npts", type=int, default=None, choices=[1, 9, 81],
                    help="operator mode: stencil points")
    ap.add_argument("--defl", type=int, default=None, metavar="NEV",
                    help="time the deflated Chebyshev coarse solve with NEV eigenvectors "
                         "(Sec. 2.3) instead of the block-CG solve")
    ap.add_argument("--defl-order", type=int, default=120)
    ap.add_argument("--defl-prec", default="fp16",
                    choices=["fp64", "df32", "fp32", "bf16", "fp16", "fp16x", "tc32"])
    ap.add_argument("--blocking", action="store_true",
                    help="time block project / promote (Sec. 2.5.1) at the Table 6 shape")
    ap.add_argument("--blocks", default="4096,256,64",
                    help="n_blocks,v_block,n_basis for --blocking (nrhs from --nrhs, default 12)")
    ap.add_argument("--block-algebra", action="store_true",
                    help="time the complex64 Gram and block update (Fig. 2) at the workload's "
                         "vector shape (V nb rows, nrhs columns), tensor-core and FMA kernels")
    ap.add_argument("--dtype", default="c128", choices=["c128", "c64"])
    ap.add_argument("--batch", default=None, choices=["uneven12", "small"],
                    help="batched solve of independent problems against one-at-a-time solves: "
                         "twelve problems of uneven L, nb and nrhs, or twelve 4^4 problems")
    ap.add_argument("--cg5d", action="store_true",
                    help="one CG on the enlarged 5D system (Sec. 2.1) against FP64 block CG")
    ap.add_argument("--coarsen", default=None, metavar="LF,BLOCK,NBF,NBASIS",
                    help="time coarsening an 81-point fine operator, e.g. 8,2,12,24: fine "
                         "lattice 8^4, 2^4 blocks, 12 fine components, 24 basis vectors")
    ap.add_argument("--twolevel", default=None, metavar="LF,NBF,EPS,MASS",
                    help="flexible ADEF2 with the variable (Krylov) two-level preconditioner "
                         "against Preconditioned BlockCGrQ with the stationary one (Fig. 1, Fig. 2 "
                         "right, Sec. 2.3) on a synthetic covariant Laplacian of mass MASS, "
                         "e.g. 16,6,0.3,0.0005")
    ap.add_argument("--tl-block", type=int, default=2, help="--twolevel: block extent")
    ap.add_argument("--tl-nbasis", type=int, default=12, help="--twolevel: basis vectors per block")
    ap.add_argument("--tl-nev", type=int, default=64, help="--twolevel: coarse eigenvectors")
    ap.add_argument("--tl-nrhs", type=int, default=12, help="--twolevel: right-hand sides")
    ap.add_argument("--tl-cheb-order", type=int, default=120,
                    help="--twolevel: order of the deflated Chebyshev coarse solve")
    ap.add_argument("--no-autotune", action="store_true",
                    help="skip the launch-shape autotuner (run before the timed region)")
    return ap.parse_args()


# ---------------------------------------------------------------- helpers
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
            except (ValueError, IndexError):
                continue
            for n, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d["hbm_gbs"], d.get("bf16_tflops"), "measured"
    except (OSError, KeyError, ValueError):
        return 6400.0, 1800.0, "fallback"


def op_flops(w, R):
    V = int(np.prod(w["L"]))
    return 8.0 * w["nb"] ** 2 * R * w["npts"] * V


def op_bytes(w, R, prec):
    """Algorithmic bytes of one application: coefficients once, input and
    output vectors once (neighbour re-reads not counted)."""
    V = int(np.prod(w["L"]))
    coef = {"fp64": 16, "df32": 16, "fp32": 8, "bf16": 4, "fp16": 4, "fp16x": 4, "tc32": 8,
            "oz": 32}[prec]
    vec = 16 if prec in WIDE else 8
    # site scale + diagonal (float pair; a double pair for the digit image)
    extra = {"fp64": 0, "df32": 0, "fp32": 0, "oz": 16 * V}.get(prec, 8 * V)
    return w["npts"] * V * w["nb"] ** 2 * coef + extra + 2 * V * w["nb"] * R * vec


def cheb_launch_bytes(w, R, prec, order):
    """Algorithmic bytes of an average preconditioner launch in the solve: the
    operator's coefficients and input, and the Chebyshev step done in its
    epilogue -- the first step writes T and P (3 vector passes with the
    input), each later one also reads T_prev and P (5 passes); W is never
    stored."""
    V = int(np.prod(w["L"]))
    vec = V * w["nb"] * R * 8
    coef_only = op_bytes(w, R, prec) - 2 * vec
    passes = (3 + 5 * (order - 1)) / order if order > 0 else 2
    return coef_only + passes * vec


# ---------------------------------------------------------------- oracle leg
class OracleSample:
    """Oracle (plain C + OpenMP, FP64) coarse operator on a sample of sites.

    The timed quantity is one application on the sampled sites, scaled to
    the whole lattice and multiplied by the FP64 block-CG application count
    (iterations + 2 residual evaluations), per RHS: the oracle's own
    time-to-solution for the plain FP64 method on this workload."""

    def __init__(self, w, shift, sites):
        from synth import coarse_op, stencil
        self.w = w
        self.disp, _ = stencil(w["npts"])
        self.V = int(np.prod(w["L"]))
        rng = np.random.default_rng(0)
        self.idx = np.sort(rng.choice(self.V, size=min(sites, self.V), replace=False))
        self.A_s = coarse_op(w["L"], w["nb"], w["npts"], w["seed"], shift, sites=self.idx)

    def ms_per_rhs(self, B_host, applications, min_seconds=10.0):
        from oracle import native
        w = self.w
        native.coarse_op_apply_sites(self.A_s[:2], B_host, w["L"], self.disp, self.idx[:2])
        # repeat the sampled application until about min_seconds of CPU work
        reps = 0
        t0 = time.perf_counter()
        while True:
            native.coarse_op_apply_sites(self.A_s, B_host, w["L"], self.disp, self.idx)
            reps += 1
            elapsed = time.perf_counter() - t0
            if elapsed >= min_seconds:
                break
        dt = elapsed / reps
        full_ms = dt * 1e3 * self.V / len(self.idx)
        R = B_host.shape[-1]
        return full_ms * applications / R, dict(
            sample=f"FP64 oracle operator on {len(self.idx)} of {self.V} sites, {reps} repetitions "
                   f"({elapsed:.1f} s, {dt:.3f} s each), scaled x{self.V / len(self.idx):.0f} to one "
                   f"application, x{applications} applications (those of the FP64 block CG)",
            full_apply_ms=full_ms,
            cores=int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1)))


def fp64_iteration_count(name):
    """Iterations the plain FP64 block CG needs on this workload, as measured
    on the GPU and recorded in profiles/fp64_block_cg_iterations.txt (used by
    the reference arm only, which runs no GPU code; our own arm measures the
    count in the same run)."""
    p = os.path.join(ROOT, "profiles", "fp64_block_cg_iterations.txt")
    try:
        with open(p) as f:
            for line in f:
                parts = line.split()
                if len(parts) >= 2 and parts[0] == name and parts[1].isdigit():
                    return int(parts[1])
    except OSError:
        pass
    return None


def dram_traffic(prec, name):
    """Measured DRAM bytes per launch of the operator kernel (ncu), from
    profiles/dram_traffic_per_launch.txt, or None if not captured."""
    p = os.path.join(ROOT, "profiles", "dram_traffic_per_launch.txt")
    try:
        with open(p) as f:
            for line in f:
                parts = line.split()
                if len(parts) >= 3 and parts[0] == prec and parts[1] == name:
                    return float(parts[2])
    except (OSError, ValueError):
        pass
    return None


def run_reference(a, w, shift):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import torch  # noqa: F401  (only to match the environment of the other arm)
    from synth import vectors
    R = w["nrhs"]
    B = vectors(w["L"], w["nb"], R, w["seed"])
    iters = fp64_iteration_count(w["name"]) or 0
    sample = OracleSample(w, shift, a.cpu_sites)
    vals = []
    for i in range(a.warmup + a.steps):
        # FP64 block CG from a zero guess: one application per iteration and
        # one for the final true residual
        v, meta = sample.ms_per_rhs(B, iters + 1)
        if i >= a.warmup:
            vals.append(v)
    val = statistics.median(vals)
    out = {"impl": "reference", "metric": METRIC, "value": val, "unit": "ms/RHS",
           "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup, "ms_per_step": val * R,
           "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": w["name"], "L": list(w["L"]), "nb": w["nb"], "npts": w["npts"],
                      "nrhs": R, "kappa": w["kappa"], "tol": 1e-8,
                      "method": "plain FP64 block CG (the oracle's operator on the host cores)"},
           "cpu_baseline": {"value": val, "unit": "ms/RHS", "cores": meta["cores"],
                            "kind": "oracle", "sample": meta["sample"]},
           "e2e": {"value": val, "unit": "ms/RHS", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0},
           "fp64_iterations": iters,
           "fp64_iterations_source": "recorded from the GPU FP64 block CG of this workload "
                                     "(profiles/fp64_block_cg_iterations.txt)"}
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------- our arm
def run_op(a, w, shift):
    """Coarse-operator throughput: K applications of the operator in one
    precision, inputs resident in HBM (coefficients far larger than L2)."""
    import torch
    import paper_2409_03904_b300 as mrhs
    import synth.device as sdev
    from synth import stencil
    over = {}
    if a.lattice:
        over["L"] = tuple(int(v) for v in a.lattice.split(","))
    for k in ("nrhs", "nb", "npts"):
        if getattr(a, k) is not None:
            over[k] = getattr(a, k)
    w = dict(w, **over)
    V, nb, prec = int(np.prod(w["L"])), w["nb"], a.op
    disp, _ = stencil(w["npts"])
    dev = torch.device("cuda", 0)
    A = sdev.coarse_op(w["L"], nb, w["npts"], w["seed"], shift, device=dev)
    op = mrhs.CoarseOp(A, w["L"], disp, (prec,))
    del A
    torch.cuda.empty_cache()
    Rs = [int(v) for v in a.nrhs_list.split(",")] if a.nrhs_list else [w["nrhs"]]

    def one(R):
        if a.nrhs_list:
            over["nrhs"] = R
        w["nrhs"] = R
        vdt = torch.complex128 if prec in WIDE else torch.complex64
        X = sdev.vectors(w["L"], nb, R, w["seed"], device=dev).to(vdt)
        Y = torch.empty_like(X)
        stream = torch.cuda.current_stream()
        tuned = None
        if not a.no_autotune and prec not in ("fp64", "fp32", "df32", "oz"):
            try:
                tuned = mrhs.autotune(op, prec, R, reps=3)
            except mrhs.MrhsError:
                tuned = None
        for _ in range(a.warmup):
            op.apply(X, prec, out=Y)
        op.kernel_timing(True)
        l0 = mrhs.launch_count()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(0) as clk:
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(a.steps):
                op.apply(X, prec, out=Y)
            e1.record(stream)
            torch.cuda.synchronize()
        launches = mrhs.launch_count() - l0
        ms = e0.elapsed_time(e1) / a.steps
        nk, kms = op.kernel_time(prec)
        op.kernel_timing(False)
        flops = op_flops(w, R)
        byts = op_bytes(w, R, prec)
        hbm, bf16_peak, kind = peaks()
        per = kms / max(nk, 1)
        roof = {"bound": "hbm", "achieved": byts / (per * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
                "frac": byts / (per * 1e-3) / 1e9 / hbm, "traffic": None,
                "kernel": f"coarse operator ({prec})", "algorithmic_bytes": byts, "launch_ms": per,
                "launches": nk, "peak_kind": f"{kind} copy bandwidth"}
        if prec == "oz":
            # digit-sliced form: bound by the fp16 tensor pipe.  Algorithmic work =
            # the 36 digit-pair products (s + t <= 9) of the complex operator;
            # issued = 20 MMAs of M = 128 per point and K step (two digit levels
            # per accumulator, 4 of the 40 half-MMAs have a zero half)
            pairs = sum(range(1, 9))
            alg = pairs * flops
            issued = 20 * 2 * 128 * (2 * ((nb + 7) // 8 * 8)) * ((nb + 15) // 16 * 16) \
                * w["npts"] * V
            roof = {"bound": "tensor", "achieved": alg / (per * 1e-3) / 1e12, "peak": bf16_peak,
                    "unit": "TFLOP/s", "frac": alg / (per * 1e-3) / 1e12 / bf16_peak,
                    "traffic": None if over else dram_traffic(prec, w["name"]), "kernel": "coarse operator (oz, tcgen05 fp16 digit MMAs)",
                    "algorithmic_flops": alg, "issued_flops": issued,
                    "issued_tflops": issued / (per * 1e-3) / 1e12,
                    "hbm_gbs": byts / (per * 1e-3) / 1e9, "launch_ms": per, "launches": nk,
                    "peak_kind": f"{kind} dense bf16 (fp16 runs at the same rate)"}
        # end to end: host input -> device, apply, device -> host result
        Xh = X.cpu().pin_memory()
        Yh = torch.empty_like(Xh).pin_memory()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(a.steps):
            Xd = Xh.to(dev, non_blocking=True)
            op.apply(Xd, prec, out=Y)
            Yh.copy_(Y, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        e2e_ms = e0.elapsed_time(e1) / a.steps
        out = {"metric": "coarse-op TFLOP/s at Nrhs=%d" % R, "value": flops / (ms * 1e-3) / 1e12,
               "unit": "TFLOP/s", "n_gpus": 1, "steps": a.steps, "warmup": a.warmup,
               "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
               "dtype": prec, "data": "synthetic",
               "config": {"workload": w["name"] + ("" if not over else " with " + ", ".join(
                              f"{k}={v}" for k, v in over.items())),
                          "L": list(w["L"]), "nb": nb, "npts": w["npts"], "nrhs": R,
                          "launch_shape": tuned,
                          "l2": f"inputs larger than L2 ({byts / 1e9:.2f} GB per application)"},
               "roofline": roof, "gpu_launches": launches, "clocks": clk.summary(),
               "e2e": {"value": flops / (e2e_ms * 1e-3) / 1e12, "unit": "TFLOP/s",
                       "h2d_bytes_per_step": Xh.numel() * Xh.element_size(),
                       "d2h_bytes_per_step": Yh.numel() * Yh.element_size()}}
        print(json.dumps(out), flush=True)

    for R in Rs:
        one(R)


def run_defl(a, w, shift):
    """Deflated Chebyshev coarse solve Q^{Cheby+defl}: K applications to the
    workload's sources.  With N <= 16384 the deflation basis is the n_ev
    lowest eigenvectors (dense H from the FP64 operator, torch.linalg.eigh)
    and the residual reduction |B - H Q B| / |B| is reported; larger
    lattices use random unit columns (the cost does not depend on them)."""
    import torch
    import paper_2409_03904_b300 as mrhs
    import synth.device as sdev
    from synth import stencil
    over = {k: getattr(a, k) for k in ("nrhs", "nb", "npts") if getattr(a, k) is not None}
    if a.lattice:
        over["L"] = tuple(int(v) for v in a.lattice.split(","))
    w = dict(w, **over)
    R, V, nb, prec, n_ev = w["nrhs"], int(np.prod(w["L"])), w["nb"], a.defl_prec, a.defl
    N = V * nb
    disp, _ = stencil(w["npts"])
    dev = torch.device("cuda", 0)
    A = sdev.coarse_op(w["L"], nb, w["npts"], w["seed"], shift, device=dev)
    op = mrhs.CoarseOp(A, w["L"], disp, tuple(dict.fromkeys(("fp64", prec))))
    del A
    torch.cuda.empty_cache()
    wide = prec in WIDE
    vdt = torch.complex128 if wide else torch.complex64
    B = sdev.vectors(w["L"], nb, R, w["seed"], device=dev)
    lam_max = op.lambda_max("fp64", 60)
    exact = N <= 16384
    if exact:
        H = torch.empty((N, N), dtype=torch.complex128, device=dev)
        for c0 in range(0, N, 64):
            c1 = min(N, c0 + 64)
            E = torch.zeros((N, c1 - c0), dtype=torch.complex128, device=dev)
            E[torch.arange(c0, c1, device=dev), torch.arange(c1 - c0, device=dev)] = 1
            H[:, c0:c1] = op.apply(E.reshape(V, nb, -1), "fp64").reshape(N, -1)
        ev, W = torch.linalg.eigh(H)
        del H
        lam = ev[:n_ev].cpu().numpy()
        U = W[:, :n_ev].contiguous().reshape(V, nb, n_ev)
        del W
        # the interval's lower end a factor of ten below the largest deflated
        # eigenvalue (Sec. 2.3's choice), so the deflated directions' rounding
        # residue sees little of the polynomial's growth below lo
        lo = float(ev[max(n_ev, 1) - 1].item()) / 10.0
        ukind = f"lowest {n_ev} eigenvectors (dense eigh)"
    else:
        g = torch.Generator(device=dev).manual_seed(w["seed"])
        U = torch.randn((N, n_ev), dtype=torch.complex128, device=dev, generator=g)
        U = (U / torch.linalg.vector_norm(U, dim=0, keepdim=True)).reshape(V, nb, n_ev)
        lo = lam_max / 1000.0
        lam = np.geomspace(lo / 50.0, lo, n_ev) if n_ev else np.zeros(0)
        ukind = f"{n_ev} random unit columns (timing only)"
    hi = 1.08 * lam_max
    U = U.to(vdt).contiguous()
    Bx = B.to(vdt)
    X = torch.empty_like(Bx)
    stream = torch.cuda.current_stream()
    for _ in range(a.warmup):
        op.defl_cheby(U, lam, Bx, lo, hi, a.defl_order, prec, out=X)
    op.kernel_timing(True)
    l0 = mrhs.launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(0) as clk:
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(a.steps):
            op.defl_cheby(U, lam, Bx, lo, hi, a.defl_order, prec, out=X)
        e1.record(stream)
        torch.cuda.synchronize()
    launches = mrhs.launch_count() - l0
    ms = e0.elapsed_time(e1) / a.steps
    nk, kms = op.kernel_time(prec)
    op.kernel_timing(False)
    per = kms / max(nk, 1)
    byts = op_bytes(w, R, prec)
    hbm, _, kind = peaks()
    quality = None
    if exact:
        r = B - op.apply(X.to(torch.complex128), "fp64")
        quality = float((torch.linalg.vector_norm(r.reshape(N, R), dim=0)
                         / torch.linalg.vector_norm(B.reshape(N, R), dim=0)).max())
    out = {"metric": "deflated Chebyshev coarse solve time per RHS", "value": ms / R,
           "unit": "ms/RHS", "n_gpus": 1, "steps": a.steps, "warmup": a.warmup,
           "ms_per_step": ms, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
           "dtype": prec, "data": "synthetic",
           "config": {"workload": w["name"] + ("" if not over else " with " + ", ".join(
                          f"{k}={v}" for k, v in over.items())),
                      "n_ev": n_ev, "deflation_basis": ukind, "lo": lo, "hi": hi,
                      "order": a.defl_order, "nrhs": R,
                      "l2": f"inputs larger than L2 ({byts / 1e9:.2f} GB per operator application)"},
           "residual_reduction": quality,
           "roofline": {"bound": "hbm", "achieved": byts / (per * 1e-3) / 1e9, "peak": hbm,
                        "unit": "GB/s", "frac": byts / (per * 1e-3) / 1e9 / hbm, "traffic": None,
                        "kernel": f"coarse operator ({prec}) in the recurrence",
                        "launch_ms": per, "launches": nk,
                        "peak_kind": f"{kind} copy bandwidth"},
           "gpu_launches": launches, "clocks": clk.summary()}
    print(json.dumps(out), flush=True)


def run_blocking(a):
    """Block project and promote (one GEMM per coarse site): K applications
    of each on a random basis, inputs resident in HBM."""
    import torch
    import paper_2409_03904_b300 as mrhs
    nblk, vb, nbasis = (int(v) for v in a.blocks.split(","))
    R = a.nrhs or 12
    dt = torch.complex128 if a.dtype == "c128" else torch.complex64
    dev = torch.device("cuda", 0)
    g = torch.Generator(device=dev).manual_seed(2409)
    B = torch.randn((nblk, vb, nbasis), dtype=dt, device=dev, generator=g)
    F = torch.randn((nblk, vb, R), dtype=dt, device=dev, generator=g)
    C = torch.randn((nblk, nbasis, R), dtype=dt, device=dev, generator=g)
    stream = torch.cuda.current_stream()
    res = {}
    es = 16 if a.dtype == "c128" else 8
    flops = 8.0 * nblk * vb * nbasis * R
    hbm, _, kind = peaks()
    for name, fn in (("project", lambda: mrhs.block_project(B, F)),
                     ("promote", lambda: mrhs.block_promote(B, C))):
        for _ in range(a.warmup):
            fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(a.steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / a.steps
        byts = es * nblk * (vb * nbasis + vb * R + nbasis * R)
        res[name] = {"ms": ms, "tflops": flops / (ms * 1e-3) / 1e12,
                     "gbs": byts / (ms * 1e-3) / 1e9, "hbm_frac": byts / (ms * 1e-3) / 1e9 / hbm}
    ms = res["project"]["ms"] + res["promote"]["ms"]
    out = {"metric": "block project + promote time", "value": ms, "unit": "ms",
           "n_gpus": 1, "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms,
           "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
           "dtype": a.dtype, "data": "synthetic",
           "config": {"workload": f"block project/promote, {nblk} blocks of {vb} x {nbasis}, "
                                  f"{R} RHS", "l2": f"basis {es * nblk * vb * nbasis / 1e9:.2f} GB"},
           "project": res["project"], "promote": res["promote"],
           "peak_kind": f"{kind} copy bandwidth"}
    print(json.dumps(out), flush=True)


def run_block_algebra(a, w):
    """The inner solve's block algebra at the workload's shape: Gram X^dagger Y
    (two blocks, and one block against itself) and the block update
    Y = Y + X M, on complex64 [V nb][R] blocks resident in HBM, each timed over
    K launches with CUDA events, for the tensor-core kernels (mode 1) and the
    FP32 FMA kernels (mode 0).  Bytes: blocks read (and written) once."""
    import torch
    import paper_2409_03904_b300 as mrhs
    nb = a.nb or w["nb"]
    R = a.nrhs or w["nrhs"]
    L = tuple(int(v) for v in a.lattice.split(",")) if a.lattice else w["L"]
    N = int(np.prod(L)) * nb
    dev = torch.device("cuda", 0)
    g = torch.Generator(device=dev).manual_seed(2409)
    X = torch.randn((N, R), dtype=torch.complex64, device=dev, generator=g)
    Y = torch.randn((N, R), dtype=torch.complex64, device=dev, generator=g)
    M = torch.randn((R, R), dtype=torch.complex128, device=dev, generator=g)
    stream = torch.cuda.current_stream()
    hbm, _, kind = peaks()
    blk = 8.0 * N * R
    cases = (("gram", lambda: mrhs.block_inner(X, Y), 2 * blk),
             ("gram_herm", lambda: mrhs.block_inner(X, X), blk),
             ("update", lambda: mrhs.block_axpy(Y, X, M, 1.0), 3 * blk))
    res = {}
    for mode in (1, 0):
        prev = mrhs.block_tc(mode)
        for name, fn, byts in cases:
            for _ in range(a.warmup):
                fn()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(a.steps):
                fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / a.steps
            res[f"{name}_{'tc' if mode else 'fma'}"] = {
                "ms": ms, "gbs": byts / (ms * 1e-3) / 1e9,
                "hbm_frac": byts / (ms * 1e-3) / 1e9 / hbm}
        mrhs.block_tc(prev)
    ms = res["gram_tc"]["ms"] + res["update_tc"]["ms"]
    out = {"metric": "block algebra time (Gram + update, tensor cores)", "value": ms,
           "unit": "ms", "n_gpus": 1, "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms,
           "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
           "dtype": "c64", "data": "synthetic",
           "config": {"workload": f"complex64 blocks of {N} x {R} (lattice {L}, nb {nb})",
                      "l2": f"each block {blk / 1e9:.2f} GB (inputs larger than L2 at the "
                            "workload shape)"},
           "kernels": res, "peak_kind": f"{kind} copy bandwidth"}
    print(json.dumps(out), flush=True)


def run_batch(a):
    """Lockstep batched mixed solve (mrhs_batch_solve) against the same
    problems solved one after another (block_cg_solve), to tol 1e-8, plus
    one batched operator application against the single ones."""
    import torch
    import paper_2409_03904_b300 as mrhs
    import synth.device as sdev
    from synth import BATCH, load_shift, stencil
    if a.batch == "uneven12":
        probs = [(w, 0) for w in BATCH]
    else:      # the four 4^4 problems of the list, three sources each
        small = [w for w in BATCH if w["L"] == (4, 4, 4, 4)]
        probs = [(w, c) for c in range(3) for w in small]
    ops, Bs = [], []
    for w, c in probs:
        disp, _ = stencil(w["npts"])
        A = sdev.coarse_op(w["L"], w["nb"], w["npts"], w["seed"], load_shift(w["name"]))
        ops.append(mrhs.CoarseOp(A, w["L"], disp, ("fp16x", "tc32", "oz")))
        del A
        Bs.append(sdev.vectors(w["L"], w["nb"], w["nrhs"], w["seed"] + 101 * c))
    for o in ops:
        o.lambda_max("fp16x", 40)

    def timed(f):
        torch.cuda.synchronize()
        t = time.perf_counter()
        r = f()
        torch.cuda.synchronize()
        return r, (time.perf_counter() - t) * 1e3

    tb, ts = [], []
    for i in range(a.warmup + a.steps):
        (Xs, infos), t1 = timed(lambda: mrhs.batch_solve(ops, Bs, tol=1e-8))
        res, t2 = timed(lambda: [o.solve(B, mode="mixed", tol=1e-8) for o, B in zip(ops, Bs)])
        if i >= a.warmup:
            tb.append(t1)
            ts.append(t2)
    Xc = [B.to(torch.complex64) for B in Bs]
    apply = {}
    for p in ("fp16x", "tc32"):
        for _ in range(3):
            mrhs.batch_apply(ops, Xc, p)
        _, t1 = timed(lambda: [mrhs.batch_apply(ops, Xc, p) for _ in range(20)])
        for _ in range(3):
            [o.apply(X, p) for o, X in zip(ops, Xc)]
        _, t2 = timed(lambda: [[o.apply(X, p) for o, X in zip(ops, Xc)] for _ in range(20)])
        apply[p] = {"batched_ms": t1 / 20, "one_by_one_ms": t2 / 20}
    nrhs = sum(int(B.shape[2]) for B in Bs)
    bt, st = statistics.median(tb), statistics.median(ts)
    out = {"metric": "batched block-CG time-to-1e-8 per RHS", "value": bt / nrhs, "unit": "ms/RHS",
           "n_gpus": 1, "steps": a.steps, "warmup": a.warmup, "ms_per_step": bt,
           "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
           "dtype": "f64+oz+tc32+fp16x", "data": "synthetic",
           "config": {"workload": f"{len(probs)} independent problems ({a.batch})",
                      "problems": [w["name"] for w, _ in probs], "nrhs_total": nrhs, "tol": 1e-8},
           "one_by_one_ms": st, "batched_over_one_by_one": st / bt,
           "iters": [i["iters"] for i in infos],
           "max_true_resid": max(max(i["resid"]) for i in infos),
           "apply": apply}
    print(json.dumps(out), flush=True)


def run_cg5d(a, w, shift):
    """Unpreconditioned FP64 solves to 1e-8 of the workload: BlockCGrQ
    (Fig. 2 left) against one CG on the enlarged five-dimensional system with
    the FP64 and the DF32 operator; iterations and wall time."""
    import torch
    import paper_2409_03904_b300 as mrhs
    import synth.device as sdev
    from synth import stencil
    R, nb = w["nrhs"], w["nb"]
    disp, _ = stencil(w["npts"])
    dev = torch.device("cuda", 0)
    A = sdev.coarse_op(w["L"], nb, w["npts"], w["seed"], shift, device=dev)
    op = mrhs.CoarseOp(A, w["L"], disp, ("fp64",))
    del A
    torch.cuda.empty_cache()
    B = sdev.vectors(w["L"], nb, R, w["seed"], device=dev)
    runs = {"block_cg_fp64": dict(mode="fp64"), "cg5d_fp64": dict(mode="cg5d"),
            "cg5d_df32": dict(mode="cg5d", krylov_prec="df32")}
    res = {}
    for name, kw in runs.items():
        for i in range(a.warmup + 1):
            X, info = op.solve(B, tol=1e-8, maxiter=20000, raise_on_fail=False, **kw)
        res[name] = {"iters": info["iters"], "ms": info["ms_total"], "ms_per_rhs": info["ms_total"] / R,
                     "max_true_resid": max(info["resid"]), "ms_per_iter": info["ms_total"] / max(info["iters"], 1)}
    out = {"metric": "unpreconditioned FP64 solve time per RHS: block CG vs 5D CG",
           "value": res["cg5d_fp64"]["ms_per_rhs"], "unit": "ms/RHS", "n_gpus": 1,
           "steps": 1, "warmup": a.warmup, "higher_is_better": False, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": w["name"], "tol": 1e-8, "nrhs": R}, "solves": res}
    print(json.dumps(out), flush=True)


def run_coarsen(a):
    """Coarse operator of a synthetic 81-point fine operator on a random
    block-orthonormal basis (momentum-phase method, 81 multi-RHS FP64 fine
    applications): K coarsenings, CUDA events."""
    import torch
    import paper_2409_03904_b300 as mrhs
    import synth.device as sdev
    from synth import stencil
    lf, blk, nbf, nbasis = (int(v) for v in a.coarsen.split(","))
    Lf, block = (lf,) * 4, (blk,) * 4
    Lc = tuple(l // b for l, b in zip(Lf, block))
    disp, _ = stencil(81)
    dev = torch.device("cuda", 0)
    A = sdev.coarse_op(Lf, nbf, 81, 2409, 6.0, device=dev)
    fine = mrhs.CoarseOp(A, Lf, disp, ("fp64",))
    del A
    Vc, vb = int(np.prod(Lc)), blk ** 4 * nbf
    g = torch.Generator(device=dev).manual_seed(2410)
    basis = torch.linalg.qr(torch.randn((Vc, vb, nbasis), dtype=torch.complex128, device=dev,
                                        generator=g))[0].contiguous()
    stream = torch.cuda.current_stream()
    for _ in range(a.warmup):
        fine.coarsen(block, basis, disp)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(a.steps):
        Ac = fine.coarsen(block, basis, disp)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / a.steps
    Vf = int(np.prod(Lf))
    fine_flops = 81 * 8.0 * nbf ** 2 * nbasis * 81 * Vf          # 81 fine applications
    proj_flops = 81 * 8.0 * vb * nbasis * nbasis * Vc            # 81 block projections
    out = {"metric": "coarsening time (81 stencil points)", "value": ms, "unit": "ms",
           "n_gpus": 1, "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms,
           "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": f"fine {Lf} x {nbf}, 81-point; blocks {block}; coarse {Lc} x {nbasis}"},
           "fine_apply_tflops": fine_flops / (ms * 1e-3) / 1e12,
           "flops_fine": fine_flops, "flops_project": proj_flops}
    print(json.dumps(out), flush=True)


def run_twolevel(a):
    """Flexible ADEF2 (Fig. 1) with the variable preconditioner of the
    original HDCG -- 7 CG iterations per column on H + Lambda, deflated CG to
    4e-2 on the coarse grid -- against Preconditioned BlockCGrQ (Fig. 2
    right) with the stationary one of Sec. 2.3 -- an order-8 Chebyshev
    smoother and the deflated Chebyshev coarse solve -- on the same
    synthetic operator, two-level hierarchy and sources, to a true relative
    residual of 1e-8.  Plain CG per column and flexible ADEF2 with the
    stationary preconditioner are timed beside them."""
    import torch
    import paper_2409_03904_b300 as mrhs
    from paper_2409_03904_b300 import twolevel as tl
    from synth import stencil
    from synth.laplace import covariant_laplacian
    lf, nbf, eps, mass = a.twolevel.split(",")
    lf, nbf, eps, mass = int(lf), int(nbf), float(eps), float(mass)
    Lf, block = (lf,) * 4, (a.tl_block,) * 4
    Lc = tuple(l // b for l, b in zip(Lf, block))
    Vf, Vc, bv = lf ** 4, int(np.prod(Lc)), a.tl_block ** 4
    R, nbasis, nev = a.tl_nrhs, a.tl_nbasis, a.tl_nev
    d9, _ = stencil(9)
    d81, _ = stencil(81)
    dev = torch.device("cuda", 0)
    t0 = time.time()
    # the covariant Laplacian, its largest eigenvalue (power method) and a
    # near-null basis by inverse iteration on random vectors; the lowest Ritz
    # value of that basis estimates lambda_min (reported only)
    g = torch.Generator(device=dev).manual_seed(2410)
    Af = torch.from_numpy(covariant_laplacian(Lf, nbf, eps, mass, 2409)).to(dev)
    fine = mrhs.CoarseOp(Af, Lf, d9, ("fp64",))
    lam_f = fine.lambda_max("fp64", 100) * 1.05
    Vn = torch.randn((Vf, nbf, nbasis), dtype=torch.complex128, device=dev, generator=g)
    for _ in range(3):
        Vn, _i = fine.solve(Vn.contiguous(), tol=1e-3, maxiter=1000, raise_on_fail=False)
        Vn = (Vn / torch.linalg.vector_norm(Vn.reshape(-1, nbasis), dim=0)).contiguous()
    Gv = mrhs.block_inner(Vn, fine.apply(Vn, "fp64"))
    Li = torch.linalg.inv(torch.linalg.cholesky(mrhs.block_inner(Vn, Vn)))
    lam_min_est = float(torch.linalg.eigvalsh(Li @ Gv @ Li.conj().T)[0].item())
    lo_s = lam_f / 46.0                          # the paper's [2, 92] smoother interval
    As = Af.clone()
    As[:, 0] += lo_s * torch.eye(nbf, dtype=torch.complex128, device=dev)
    shifted = mrhs.CoarseOp(As, Lf, d9, ("fp64",))
    del As
    # the near-null basis cut into blocks and orthonormalised block by block
    ib = torch.stack(torch.meshgrid(*[torch.arange(b) for b in block], indexing="ij"), -1)
    ib = ib.permute(3, 2, 1, 0, 4).reshape(-1, 4)          # first direction fastest
    cc = torch.stack(torch.meshgrid(*[torch.arange(c) for c in Lc], indexing="ij"), -1)
    cc = cc.permute(3, 2, 1, 0, 4).reshape(-1, 4)
    gsite = cc[:, None, :] * torch.tensor(block) + ib[None]
    Lt = torch.tensor(Lf)
    site = gsite[..., 0] + Lt[0] * (gsite[..., 1] + Lt[1] * (gsite[..., 2] + Lt[2] * gsite[..., 3]))
    basis = Vn[site.reshape(-1).to(dev)].reshape(Vc, bv * nbf, nbasis)
    basis = torch.linalg.qr(basis)[0].contiguous()
    Ac = fine.coarsen(block, basis, d81)
    coarse = mrhs.CoarseOp(Ac, Lc, d81, ("fp64",))
    Nc = Vc * nbasis
    Hd = torch.empty((Nc, Nc), dtype=torch.complex128, device=dev)
    for c0 in range(0, Nc, 64):
        c1 = min(Nc, c0 + 64)
        E = torch.zeros((Nc, c1 - c0), dtype=torch.complex128, device=dev)
        E[torch.arange(c0, c1, device=dev), torch.arange(c1 - c0, device=dev)] = 1
        Hd[:, c0:c1] = coarse.apply(E.reshape(Vc, nbasis, -1), "fp64").reshape(Nc, -1)
    ev, W = torch.linalg.eigh(Hd)
    del Hd
    U = W[:, :nev].contiguous().reshape(Vc, nbasis, nev)
    lam = ev[:nev].cpu().numpy()
    lam_c = float(ev[-1].item()) * 1.05
    setup_s = time.time() - t0
    T = tl.Transfer(Lf, block, nbf, basis)
    two = tl.TwoLevel(fine, T, coarse)
    co = a.tl_cheb_order
    stat = two.stationary((lo_s, lam_f, 8), (U, lam, lam[-1] / 10.0, lam_c, co))
    kry = two.krylov(shifted, 7, U, lam, 4e-2)
    Qk = lambda v: two.Q(v, two.deflated_cg_solve(U, lam, 4e-2))  # noqa: E731
    Qs = lambda v: two.Q(v, two.defl_cheby_solve(U, lam, lam[-1] / 10.0, lam_c, co))  # noqa
    B = torch.randn((Vf, nbf, R), dtype=torch.complex128, device=dev, generator=g)
    runs = {
        "flex_adef2_krylov": lambda: tl.flex_adef2(two.H, kry, Qk, B, tol=1e-8, maxiter=500),
        "prec_block_cg_stationary": lambda: tl.prec_block_cg(two.H, stat, B, tol=1e-8,
                                                             maxiter=500),
        "flex_adef2_stationary": lambda: tl.flex_adef2(two.H, stat, Qs, B, tol=1e-8, maxiter=500),
        "cg_per_column": lambda: (tl.cg_columns(two.H, B, tol=1e-8, maxiter=20000,
                                                stats=cg_stats), cg_stats),
    }
    cg_stats = {}
    res = {}
    for name, f in runs.items():
        for _ in range(max(a.warmup, 1) if name != "cg_per_column" else 1):
            f()
        ms = []
        for _ in range(a.steps):
            torch.cuda.synchronize()
            t = time.perf_counter()
            X, info = f()
            torch.cuda.synchronize()
            ms.append((time.perf_counter() - t) * 1e3)
        r = B - two.H(X)
        true = (torch.linalg.vector_norm(r.reshape(-1, R), dim=0)
                / torch.linalg.vector_norm(B.reshape(-1, R), dim=0)).max().item()
        entry = {"ms": statistics.median(ms), "ms_per_rhs": statistics.median(ms) / R,
                 "max_true_resid": true}
        if info is not None:
            entry["iters"] = info["iters"]
            if "col_iters" in info:
                entry["col_iters"] = info["col_iters"]
        res[name] = entry
    out = {"metric": "two-level outer solve time per RHS: flexible ADEF2 (variable "
                     "preconditioner) vs Preconditioned BlockCGrQ (stationary)",
           "value": res["prec_block_cg_stationary"]["ms_per_rhs"], "unit": "ms/RHS",
           "n_gpus": 1, "steps": a.steps, "warmup": a.warmup, "higher_is_better": False,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": f"covariant Laplacian {Lf} x {nbf}, eps {eps}, mass {mass:g} "
                                  f"(lambda_max {lam_f / 1.05:.4g}, lowest Ritz value of the "
                                  f"basis {lam_min_est:.4g}); "
                                  f"blocks {block}, {nbasis} basis vectors, coarse {Lc}, "
                                  f"{nev} coarse eigenvectors; {R} RHS; tol 1e-8",
                      "smoother_stationary": f"Chebyshev order 8 on [{lo_s:.4g}, {lam_f:.4g}]",
                      "smoother_krylov": f"7 CG iterations per column on H + {lo_s:.4g}",
                      "coarse_stationary": f"deflated Chebyshev order {co} on "
                                           f"[{lam[-1] / 10:.4g}, {lam_c:.4g}]",
                      "coarse_krylov": "CG per column from the deflated start to 4e-2",
                      "setup_s": setup_s},
           "solves": res,
           "iteration_ratio": res["flex_adef2_krylov"]["iters"]
           / max(res["prec_block_cg_stationary"]["iters"], 1),
           "time_ratio": res["flex_adef2_krylov"]["ms"] / res["prec_block_cg_stationary"]["ms"]}
    print(json.dumps(out), flush=True)


def main():
    a = parse()
    from synth import WORKLOADS, load_shift
    w = WORKLOADS[a.workload]
    shift = load_shift(a.workload)
    if a.impl == "reference":
        return run_reference(a, w, shift)
    if a.op:
        return run_op(a, w, shift)
    if a.defl is not None:
        return run_defl(a, w, shift)
    if a.blocking:
        return run_blocking(a)
    if a.block_algebra:
        return run_block_algebra(a, w)
    if a.batch:
        return run_batch(a)
    if a.cg5d:
        return run_cg5d(a, w, shift)
    if a.coarsen:
        return run_coarsen(a)
    if a.twolevel:
        return run_twolevel(a)

    import torch
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    import paper_2409_03904_b300 as mrhs
    import synth.device as sdev
    from synth import stencil
    dev = torch.device("cuda", local)
    if a.lattice:      # a smaller lattice with the same per-site work (profiling captures)
        w = dict(w, L=tuple(int(v) for v in a.lattice.split(",")))
        w["name"] = w["name"] + " with L=" + a.lattice
    R, V, nb = w["nrhs"], int(np.prod(w["L"])), w["nb"]
    disp, _ = stencil(w["npts"])

    t0 = time.time()
    A = sdev.coarse_op(w["L"], nb, w["npts"], w["seed"], shift, device=dev)
    # the solve's operator holds the precisions the solve uses (at 12^4, nb 48:
    # digit image 124 GB, TC32 31 GB, FP16 16 GB; the FP64 copy, 62 GB, only
    # when the FP64 pipes are asked for); the others are timed afterwards on a
    # second operator
    need64 = a.fp64_op == "fp64" or a.residual in ("fp64", "df32")
    precs = tuple(dict.fromkeys((a.fp64_op, a.residual, a.precond, a.krylov)
                                + (("fp64", "df32") if need64 else ())))
    other_precs = tuple(p for p in ("fp64", "fp32", "bf16", "fp16") if p not in precs)
    op = mrhs.CoarseOp(A, w["L"], disp, precs)
    del A
    torch.cuda.empty_cache()
    B = sdev.vectors(w["L"], nb, R, w["seed"] + 7919 * rank + a.rhs_offset, device=dev)
    setup_s = time.time() - t0
    lam = op.lambda_max(a.precond, 40)
    hi = 1.08 * lam
    params = dict(mode="mixed", tol=1e-8, precond=1, precond_prec=a.precond,
                  krylov_prec=a.krylov,
                  cheb_order=a.cheb_order, cheb_hi=hi, cheb_lo=hi / a.cheb_ratio,
                  inner_tol=a.inner_tol, inner_tol_later=a.inner_tol_later,
                  maxiter=20000, max_cycles=20,
                  check_every=a.check_every, residual_prec=a.residual, recycle=a.recycle,
                  fp64_prec=a.fp64_op)

    stream = torch.cuda.current_stream()
    # launch shapes of the two tensor-core forms, tuned once for this shape
    tuned = {}
    if not a.no_autotune:
        for p in dict.fromkeys((a.precond, a.krylov)):
            if p in ("fp16x", "fp16", "bf16", "tc32"):
                try:
                    tuned[p] = mrhs.autotune(op, p, R, reps=3)
                except mrhs.MrhsError:
                    pass
    for _ in range(a.warmup):
        X, info = op.solve(B, **params)
    # ---------------- timed region: K complete solves
    op.kernel_timing(True)
    launches0 = mrhs.launch_count()      # library kernels before the timed region
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    infos = []
    with ClockSampler(local) as clk:
        barrier()
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(a.steps):
            X, info = op.solve(B, **params)
            infos.append(info)
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier()
    launches = mrhs.launch_count() - launches0
    ms = ev0.elapsed_time(ev1)
    kt = {p: op.kernel_time(p) for p in precs}
    op.kernel_timing(False)
    if world > 1:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    ms_step = ms / a.steps
    value = ms_step / (R * world)
    resid = max(max(i["resid"]) for i in infos)

    # ---------------- dominant kernel roofline (live, from the timed region)
    hbm, bf16_peak, peak_kind = peaks()
    n16, ms16 = kt[a.precond]
    roof = None
    if n16:
        per = ms16 / n16
        byts = cheb_launch_bytes(w, R, a.precond, a.cheb_order)
        ach = byts / (per * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
                "frac": ach / hbm, "traffic": dram_traffic(a.precond + "+cheb", w["name"]),
                "kernel": f"tcgen05 {a.precond} coarse operator with the Chebyshev step in its epilogue",
                "algorithmic_bytes": byts, "launch_ms": per, "launches": n16,
                "peak_kind": f"{peak_kind} copy bandwidth"}

    extras = {}
    if not a.no_extras and rank == 0:
        # standalone coarse-operator throughput at this RHS count, per precision
        cop = {}

        def time_ops(o, ps):
            for p in ps:
                Xp = B if p in WIDE else B.to(torch.complex64)
                reps = 2 if p in ("fp64", "df32", "fp32") else 10
                o.apply(Xp, p)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(reps):
                    o.apply(Xp, p)
                e1.record(stream)
                torch.cuda.synchronize()
                t = e0.elapsed_time(e1) / reps
                cop[p] = {"ms": t, "tflops": op_flops(w, R) / (t * 1e-3) / 1e12,
                          "gbs": op_bytes(w, R, p) / (t * 1e-3) / 1e9}
        time_ops(op, precs)
        extras["coarse_op"] = cop
        if "oz" in cop:
            # the FP64 operator's roofline on FP64 algorithmic bytes (complex128
            # coefficients and vectors), and on the tensor pipe it runs on
            t = cop["oz"]["ms"]
            b64 = op_bytes(w, R, "fp64")
            pairs = sum(range(1, 9))
            hbm, bf16_peak, kind = peaks()
            cop["oz"]["fp64_roofline"] = {
                "bound": "tensor", "fp64_algorithmic_bytes": b64,
                "fp64_bytes_gbs": b64 / (t * 1e-3) / 1e9,
                "fp64_bytes_hbm_frac": b64 / (t * 1e-3) / 1e9 / hbm,
                "digit_pair_tflops": pairs * op_flops(w, R) / (t * 1e-3) / 1e12,
                "tensor_frac": pairs * op_flops(w, R) / (t * 1e-3) / 1e12 / bf16_peak,
                "peak_kind": f"{kind} copy bandwidth / dense bf16"}
        # plain FP64 block CG (Fig. 2 left) to the same tolerance on the same
        # sources, run to the end once, with the FP64 operator of the solve
        Xf, fi = op.solve(B, tol=1e-8, maxiter=20000, raise_on_fail=False, fp64_prec=a.fp64_op)
        n_fp64_apply = fi["applies"][a.fp64_op]
        fp64 = {"iters": fi["iters"], "ms": fi["ms_total"], "resid": max(fi["resid"]),
                "ms_per_rhs": fi["ms_total"] / R, "operator": a.fp64_op,
                "operator_applications": n_fp64_apply, "extrapolated": False,
                "status": fi["status"]}
        del Xf
        extras["fp64_solve"] = fp64
        extras["mixed_speedup_vs_fp64"] = fp64["ms_per_rhs"] / value
        # end to end through the public API with host buffers
        Bh = B.cpu().pin_memory()
        Xh = torch.empty_like(Bh).pin_memory()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(a.steps):
            Bd = Bh.to(dev, non_blocking=True)
            Xd, _i = op.solve(Bd, **params)
            Xh.copy_(Xd, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        e2e_ms = e0.elapsed_time(e1) / a.steps
        extras["e2e"] = {"value": e2e_ms / R, "unit": "ms/RHS",
                         "h2d_bytes_per_step": Bh.numel() * 16, "d2h_bytes_per_step": Xh.numel() * 16}
        # CPU oracle on a bounded sample of the same workload, times the FP64
        # block CG's operator applications measured above
        cpu_v, meta = OracleSample(w, shift, a.cpu_sites).ms_per_rhs(Bh.numpy(), n_fp64_apply)
        extras["cpu_baseline"] = {"value": cpu_v, "unit": "ms/RHS",
                                  "cores": meta["cores"], "kind": "oracle",
                                  "sample": meta["sample"] + " (application count of the FP64 "
                                            "block CG measured in this run)",
                                  "full_apply_ms": meta["full_apply_ms"]}
        # the remaining precisions' operator throughput, on an operator of their own
        if other_precs:
            del op
            torch.cuda.empty_cache()
            A2 = sdev.coarse_op(w["L"], nb, w["npts"], w["seed"], shift, device=dev)
            op2 = mrhs.CoarseOp(A2, w["L"], disp, other_precs)
            del A2
            torch.cuda.empty_cache()
            time_ops(op2, other_precs)
            if "fp64" in other_precs and a.fp64_native_iters > 0:
                # FP64 block CG on the FP64 pipes: its cost per iteration (two
                # short runs, so start-up and final residual cancel) times the
                # iteration count measured above -- context, not the baseline
                _, f1 = op2.solve(B, tol=1e-30, maxiter=2, raise_on_fail=False, fp64_prec="fp64")
                _, f2 = op2.solve(B, tol=1e-30, maxiter=2 + a.fp64_native_iters,
                                  raise_on_fail=False, fp64_prec="fp64")
                per_it = (f2["ms_total"] - f1["ms_total"]) / max(f2["iters"] - f1["iters"], 1)
                extras["fp64_native_solve_estimate"] = {
                    "ms_per_iter": per_it, "iters": fp64["iters"], "extrapolated": True,
                    "ms_per_rhs": (per_it * fp64["iters"] + f1["ms_total"] - 2 * per_it) / R,
                    "note": "FP64-pipe operator: per-iteration time measured in this run x the "
                            "iteration count of the FP64 block CG above"}
            del op2

    if rank == 0:
        inf = infos[-1]
        out = {"metric": METRIC, "value": value, "unit": "ms/RHS", "n_gpus": world,
               "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms_step,
               "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
               "dtype": f"f64+{a.fp64_op}+{a.residual}+{a.krylov}+{a.precond}", "data": "synthetic",
               "config": {"workload": w["name"], "L": list(w["L"]), "nb": nb, "npts": w["npts"],
                          "nrhs": R, "kappa": w["kappa"], "tol": 1e-8,
                          "precond": f"chebyshev deg {a.cheb_order} {a.precond} on "
                                     f"[{hi / a.cheb_ratio:.4g}, {hi:.4g}]",
                          "inner_tol": a.inner_tol, "inner_tol_later": a.inner_tol_later,
                          "recycle": a.recycle,
                          "check_every": a.check_every,
                          "parallelism": f"replicas x{world}",
                          "residuals": f"{a.residual} per cycle, the FP64 operator "
                                       f"({a.fp64_op}) for the one that meets tol",
                          "fp64_operator": a.fp64_op,
                          "block_algebra": "inner block CG on complex64 vectors: Grams and "
                                           "block updates on the tensor cores (tcgen05) from "
                                           "exact three-term bf16 splits, six products summed "
                                           "in FP32; a Gram's FP32 sums (at most 512 rows) "
                                           "added into double-float pairs (about 2^-48) per "
                                           "CTA, the CTAs' partials summed in FP64 in a fixed "
                                           "order; Cholesky, inverses and the outer update in "
                                           "FP64",
                          "launch_shapes": tuned,
                          "l2": "inputs larger than L2 (coefficients "
                                f"{op_bytes(w, R, a.precond) / 1e9:.1f} GB per application)"},
               "solve": {"iters": inf["iters"], "cycles": inf["cycles"], "applies": inf["applies"],
                         "cycle_iters": inf["cycle_iters"], "cycle_resid": inf["cycle_resid"],
                         "cycle_flag": inf["cycle_flag"],
                         "recycle_blocks": inf["recycle_blocks"],
                         "recycle_projections": inf["recycle_projections"],
                         "max_true_resid": resid, "lambda_max_est": lam, "setup_s": setup_s},
               "roofline": roof, "gpu_launches": launches, "launches_before_timed": launches0,
               "clocks": clk.summary(),
               "kernel_time_ms": {p: {"launches": n, "ms": t} for p, (n, t) in kt.items()}}
        out.update(extras)
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
