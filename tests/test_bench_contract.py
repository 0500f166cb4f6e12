"""The JSON line bench.py prints: every key of the benchmark contract, with
the types and values the contract fixes.  The reference arm (the CPU oracle
on bounded samples) runs here on the CPU; our arm needs a GPU (marker: gpu).
Both run on the 24^3 stand-in of the 3-D workload so they finish quickly."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_bench(*argv):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *argv], cwd=ROOT,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    return json.loads(lines[0])


def check_common(d, steps, warmup):
    assert d["metric"].startswith("time-to-1e-10 residual")
    assert d["unit"] == "ms" and d["higher_is_better"] is False
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["n_gpus"] == 1 and d["steps"] == steps and d["warmup"] == warmup
    assert d["scaling"] == "weak" and d["vs_baseline"] is None
    assert d["data"] == "synthetic" and d["dtype"] in ("f32", "f64")
    assert d["config"]["workload"] == "convdiff3d_24"
    e = d["e2e"]
    assert e["unit"] == "ms" and e["value"] > 0
    assert e["h2d_bytes_per_step"] >= 0 and e["d2h_bytes_per_step"] >= 0


def test_reference_arm_line():
    d = run_bench("--impl", "reference", "--workload", "convdiff3d_24", "--steps", "1",
                  "--warmup", "0")
    check_common(d, 1, 0)
    assert d["impl"] == "reference"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["cpu"]
    assert cb["host_cores"] >= cb["cores"]
    assert cb["value"] == d["value"] and d["e2e"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0


@pytest.mark.gpu
def test_our_arm_line(gpulib):
    d = run_bench("--workload", "convdiff3d_24", "--steps", "3", "--warmup", "3",
                  "--compare-steps", "0", "--no-cpu-baseline")
    check_common(d, 3, 3)
    assert "impl" not in d or d["impl"] != "reference"
    n = d["config"]["n"]
    # inputs to the device and the solution back, every step
    assert d["e2e"]["h2d_bytes_per_step"] >= 8 * n and d["e2e"]["d2h_bytes_per_step"] >= 8 * n
    r = d["roofline"]
    assert r["bound"] in ("hbm", "tensor", "alu", "latency") and r["unit"] in ("GB/s", "TFLOP/s")
    assert r["achieved"] > 0 and r["peak"] > 0
    assert abs(r["frac"] - r["achieved"] / r["peak"]) <= 1e-3
    assert "traffic" in r
    c = d["clocks"]
    assert c["sm_max_mhz"] is None or c["sm_max_mhz"] > 0
    assert isinstance(c["reasons"], list)
    assert d["gpu_launches"] > 0
    assert d["relres"] <= 1e-10


def test_reference_arm_under_torchrun():
    """Launched as the driver launches it for N > 1 (torchrun, 127.0.0.1):
    rank 0 alone runs the oracle and prints the one line; the other rank
    exits 0 without work."""
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    r = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1",
                        "--nproc-per-node", "2", "--master-addr", "127.0.0.1",
                        "--master-port", str(port), os.path.join(ROOT, "bench.py"),
                        "--impl", "reference", "--workload", "convdiff3d_24", "--steps", "1",
                        "--warmup", "0", "--gpus", "2"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
