"""bench.py prints one JSON line with the keys the benchmark contract names:
the reference arm (the oracle on the host cores) on the CPU, and a small run
of the GPU arm on a GB300."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(args, timeout):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT,
                       capture_output=True, text=True, timeout=timeout)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    return json.loads(lines[0])


def test_reference_arm_line():
    b = _run(["--impl", "reference", "--steps", "2", "--warmup", "1"], 600)
    assert b["impl"] == "reference" and b["metric"] == "coupled-step MLUPS"
    assert b["unit"] == "MLUPS" and b["higher_is_better"] is True and b["value"] > 0
    assert b["n_gpus"] == 1 and b["steps"] == 2 and b["warmup"] == 1
    cb = b["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == b["value"]
    assert isinstance(cb["sample"], str) and cb["sample"]
    e = b["e2e"]
    assert e["value"] == b["value"] and e["unit"] == b["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0
    assert "workload" in b["config"]


@pytest.mark.gpu
def test_gpu_arm_line():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    b = _run(["--ncases", "16", "--steps", "5", "--warmup", "3", "--no-extras",
              "--cpu-seconds", "2"], 900)
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "roofline", "clocks", "gpu_launches", "e2e", "cpu_baseline"):
        assert k in b, k
    assert b["n_gpus"] == 1 and b["steps"] == 5 and b["warmup"] == 3 and b["value"] > 0
    # per step and chain a step kernel and a volume finalisation, one clock
    # kernel per graph of up to 64 steps
    nch = b["config"]["chains"]
    assert b["scaling"] == "weak" and b["dtype"] == "f32" and b["gpu_launches"] == 2 * nch * 5 + 1
    r = b["roofline"]
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["peak"] > 0
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-3
    assert set(b["clocks"]) >= {"sm_mhz", "sm_max_mhz", "reasons"}
    e = b["e2e"]
    assert e["unit"] == "MLUPS" and e["value"] > 0
    assert e["h2d_bytes_per_step"] > 0 and e["d2h_bytes_per_step"] == 16 * 8
    cb = b["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] > 0
    assert "workload" in b["config"]
