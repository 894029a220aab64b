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
    allc = cb["all_cores"]             # the oracle on every host core beside the one-core rate
    assert allc["cores"] >= 1 and allc["value"] > 0 and allc["unit"] == line["unit"]
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


def _bench_module():
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


PEAKS = {"hbm_gbs": 6777.6, "sm_max_mhz": 2070.0}
ALU_PEAK_T = 152 * 128 * 2070e6 / 1e12          # FP32 lanes x clock


def test_roofline_fused_fp32_kite():
    """The reported roofline of the fused FP32 kernel: 54 operations per pair
    over n^2 pairs per launch, divided by the average launch time, against
    the lane peak; traffic from the ncu table for this exact configuration
    (null while no capture of the current kernel is recorded)."""
    b = _bench_module()
    n, ms, launches = 32768, 37.0, 10
    spec = {"nrhs": 64, "bc": "soft", "precision": "fp32", "curve": "kite"}
    r = b.kernel_rooflines({"matvec_fp32": (ms, launches)}, spec, {"matvec_variant": 2},
                           PEAKS, "measured", n, 1)["matvec_fp32"]
    want = 54 * n * n / (ms / 1e3 / launches) / 1e12
    assert abs(r["achieved"] - want) < 1e-9 * want
    assert abs(r["frac"] - want / ALU_PEAK_T) < 1e-12
    assert r["bound"] == "alu"
    # with the matvec count known, the work is per matvec, not per launch
    # (a sound-hard tensor-core matvec takes an S and a D' launch)
    spec_h = {"nrhs": 4, "bc": "hard", "precision": "fp32", "curve": "star"}
    rh = b.kernel_rooflines({"matvec_fp32": (20.0, 10)}, spec_h,
                            {"matvec_variant": 2, "inner_matvecs": 5}, PEAKS, "measured", n, 1)
    want_h = (36 + 42) * n * n / (20.0 / 1e3 / 5) / 1e12
    assert abs(rh["matvec_fp32"]["achieved"] - want_h) < 1e-9 * want_h
    key = ("matvec_fp32", "kite", n, 64, 2)
    assert r["traffic"] == b.NCU_TRAFFIC.get(key)


@pytest.mark.parametrize("bc,variant,ops", [
    ("soft", 1, 563 + 48 * 5), ("hard", 1, 548 + 4 * 48 * 5),
    ("soft", 2, 563 + 48), ("hard", 2, 470 + 509 + 2 * 48)])
def test_roofline_double_float_residual(bc, variant, ops):
    """Residual kernels: the double-float entry (sound hard: S and D' from one
    phase on the CUDA cores, in two passes on the tensor cores) plus the
    per-right-hand-side Dot2 sums (4 sums per RHS for sound hard) or the
    slicing."""
    b = _bench_module()
    n, ms = 4096, 8.0
    spec = {"nrhs": 5, "bc": bc, "precision": "fp32", "curve": "star"}
    r = b.kernel_rooflines({"matvec_fp64": (ms, 2)}, spec, {"residual_variant": variant},
                           PEAKS, "measured", n, 1)["matvec_fp64"]
    want = ops * n * n / (ms / 1e3 / 2) / 1e12
    assert abs(r["achieved"] - want) < 1e-9 * want and r["unit"] == "Top/s"
    assert r["traffic"] is None


def test_roofline_stored_and_arnoldi():
    b = _bench_module()
    n = 1000
    spec = {"nrhs": 32, "bc": "soft", "precision": "tensor", "curve": "star"}
    kt = {"matvec_tensor": (2.0, 4), "arnoldi": (3.0, 100)}
    stats = {"arnoldi_elems": 7_000_000, "basis_fp32": True}
    r = b.kernel_rooflines(kt, spec, stats, PEAKS, "measured", n, 2)
    pitch = 1024                                  # n rounded up to 64
    want = n * pitch * 8 / (2.0 / 1e3 / 4) / 1e9
    assert abs(r["matvec_tensor"]["achieved"] - want) < 1e-9 * want
    assert abs(r["matvec_tensor"]["frac"] - want / 6777.6) < 1e-12
    want = 4 * 7_000_000 * 2 * 8 / 3e-3 / 1e9     # four passes, 8-byte elements, 2 solves
    assert abs(r["arnoldi"]["achieved"] - want) < 1e-9 * want


def test_measured_peaks_are_read():
    b = _bench_module()
    peaks, src = b.measured_peaks()
    if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")):
        assert src == "measured" and peaks["hbm_gbs"] > 1000
    else:
        assert src == "fallback" and peaks["hbm_gbs"] == 6800.0


def test_reference_specs_of_the_batch_sample_the_oracle():
    """The batch workload's oracle sample (four of its stars) carries the
    coupling eta = omega the oracle's rows need."""
    import argparse
    bench = _bench_module()
    args = argparse.Namespace(workload="stars", count=256, precision=None, n=None, nrhs=None,
                              eta_factor=None)
    specs = bench.reference_specs(args)
    assert len(specs) == 4
    for sp in specs:
        assert sp["eta"] == sp["omega"]
    pairs, secs = bench.oracle_sample(specs[0], 2)
    assert pairs == 2 * specs[0]["n"] and secs > 0


def test_other_configs_only_after_the_plain_headline():
    """The default run appends the brief runs of the other configurations;
    any override of the headline (another workload, n, precision, solver
    option) or --no-extras turns them off."""
    b = _bench_module()
    assert b.default_headline(_args(b, []))
    for extra in (["--no-extras"], ["--workload", "star"], ["--n", "8192"], ["--block"],
                  ["--precision", "fp64"], ["--fp64-basis"], ["--rtol", "1e-6"]):
        assert not b.default_headline(_args(b, extra)), extra


def _args(b, argv):
    old = sys.argv
    try:
        sys.argv = ["bench.py"] + argv
        return b.parse()
    finally:
        sys.argv = old


def test_brief_summary_of_a_run():
    b = _bench_module()
    run = {"metric": "m", "value": 2.0, "unit": "u", "steps": 3, "warmup": 3, "ms_per_step": 5.0,
           "config": {"workload": "w"}, "kernel_ms": {"x": 1.0},
           "roofline": {"bound": "hbm", "achieved": 1.0, "peak": 2.0, "unit": "GB/s", "frac": 0.5,
                        "traffic": None}}
    out = b._brief(run)
    assert out["workload"] == "w" and out["value"] == 2.0 and "kernel_ms" not in out
    assert out["roofline"]["frac"] == 0.5 and "traffic" not in out["roofline"]
