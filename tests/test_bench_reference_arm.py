"""bench.py's reference arm, as launched for N > 1: under torchrun with two
ranks, rank 0 alone times the oracle on the host cores and prints one JSON
line; the other rank exits 0 without work. The line carries the keys the
benchmark contract asks of that arm. CPU only; about half a minute."""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_reference_arm_under_torchrun_prints_one_line():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           "bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "1"]
    out = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, out.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and (d["steps"], d["warmup"]) == (1, 1)
    assert d["metric"] and d["unit"] == "ms/RHS" and d["higher_is_better"] is False
    assert d["value"] > 0 and d["config"]["workload"] == "L12_nb48_81pt_r32"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "ms/RHS", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
