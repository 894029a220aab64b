"""The benchmark's output contract on the CPU: the reference arm (the oracle,
timed on host cores) prints one JSON line with the keys the driver reads, and
our arm fails loudly, instead of falling back to the CPU, when no GPU is
present."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(args, timeout=600):
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, cwd=ROOT,
                          capture_output=True, text=True, timeout=timeout)


def test_reference_arm_prints_the_contract_line():
    r = _run(["--impl", "reference", "--workload", "disk", "--steps", "1", "--warmup", "1"])
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "dtype", "data", "config"):
        assert key in line, key
    assert line["value"] > 0 and line["steps"] == 1 and line["warmup"] == 1
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and isinstance(cb["sample"], str)
    assert cb["value"] == line["value"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
    assert "workload" in line["config"]


def test_our_arm_needs_a_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    r = _run(["--steps", "1", "--warmup", "3"], timeout=300)
    assert r.returncode != 0
    assert "NVIDIA" in r.stderr or "CUDA" in r.stderr or "cuda" in r.stderr


def test_reference_arm_coupling_option():
    """--eta-factor sets eta = factor x omega for the single-operator
    workloads and says so in the config; the batch workloads refuse it."""
    r = _run(["--impl", "reference", "--workload", "disk", "--steps", "1", "--warmup", "1",
              "--eta-factor", "0.5"])
    assert r.returncode == 0, r.stderr[-2000:]
    cfg = json.loads(r.stdout.strip().splitlines()[-1])["config"]
    assert cfg["eta"] == 0.5 * cfg["omega"] and "eta=0.5*omega" in cfg["workload"]
    r = _run(["--impl", "reference", "--workload", "stars", "--eta-factor", "0.5"], timeout=120)
    assert r.returncode != 0 and "single-operator" in r.stderr
