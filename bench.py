"""Benchmark of the CFIE hot path on one GB300 (or N independent replicas).

A step is one pass of the whole path over one batch of synthetic input:
sample the curve and build the Kress tables (cfie_discretise), form the
plane-wave right-hand sides (cfie_rhs_plane_waves) and solve all of them with
GMRES (cfie_gmres_solve) to the target accuracy.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload kite|star|disk] [--precision fp32|fp64]

Metric: CFIE kernel-pair evaluations per second, where one kernel-pair
evaluation is the evaluation of the Nystrom kernel for one (target, source)
pair inside one block matvec (shared by all right-hand sides of the block).
Solves per second (one solve = one right-hand side at the target accuracy) are
reported beside it.

Multi-GPU: replicas only (one independent workload per rank, no collective on
the data path); value = pair evaluations of all ranks / max-over-ranks time.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "CFIE kernel-pair evals/s"
UNIT = "pair-evals/s"
SERVE_METRIC = "CFIE solves/s at 1e-8 residual (served; p50/p99 latency beside it)"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="kite",
                   choices=["kite", "star", "disk", "stars", "serve", "ellipse", "ellipse-hard"])
    p.add_argument("--precision", default=None, choices=["fp32", "fp64", "tensor", None])
    p.add_argument("--count", type=int, default=None,
                   help="stars: operators in the batch (256); serve: requests (32)")
    p.add_argument("--rtol", type=float, default=None)
    p.add_argument("--n", type=int, default=None, help="override the workload's n (profiling)")
    p.add_argument("--nrhs", type=int, default=None, help="override the number of directions")
    p.add_argument("--eta-factor", type=float, default=None,
                   help="coupling eta = factor x omega for the single-operator workloads (default 1)")
    p.add_argument("--dirprec", action="store_true",
                   help="single-operator sound-soft workloads: nodes equispaced in arclength "
                        "(n = 4^q p, p = 8) and the directional preconditioner of Section 2 on "
                        "the right of every solve (its setup inside each step)")
    p.add_argument("--block", action="store_true",
                   help="single-operator workloads: one block GMRES over all right-hand sides "
                        "(restart in block steps: 40) instead of one GMRES per right-hand side")
    p.add_argument("--fp64-basis", action="store_true",
                   help="refined precisions: FP64 inner Krylov basis instead of FP32")
    p.add_argument("--serve-batch", type=int, default=8,
                   help="serve: requests a free slot takes at once and solves as one batch")
    p.add_argument("--serve-slots", type=int, default=8, help="serve: concurrent slots")
    p.add_argument("--serve-block-min", type=int, default=8,
                   help="serve: requests with at least this many directions and --serve-block-min-n "
                        "nodes use block GMRES (0: off)")
    p.add_argument("--serve-block-min-n", type=int, default=16384)
    p.add_argument("--serve-stored-max-n", type=int, default=16384,
                   help="serve: sound-soft requests up to this n use the stored tensor-core form")
    p.add_argument("--no-extras", action="store_true",
                   help="headline workload only: skip the short runs of the other configurations "
                        "that the default run appends (other_configs)")
    p.add_argument("--oracle-budget", type=float, default=None, help=argparse.SUPPRESS)
    return p.parse_args()


# ---------------------------------------------------------------------------
# workload definitions (shapes from inputs.WORKLOADS)
# ---------------------------------------------------------------------------
def workload(name, precision, n=None, nrhs=None, eta_factor=None):
    from paper_1408_1578_gb300 import inputs
    spec = dict(inputs.WORKLOADS[name])
    spec["name"] = name
    if n:
        # same points per wavelength as the full workload
        spec["omega"] = spec["omega"] * n / spec["n"]
        spec["n"] = n
        spec["name"] = f"{name} (reduced n={n})"
    if nrhs:
        spec["nrhs"] = nrhs
    # Section 1 asks only for eta = O(omega)
    spec["eta_factor"] = eta_factor or 1.0
    spec["eta"] = spec["eta_factor"] * spec["omega"]
    if precision is None:
        precision = "fp32" if name in ("kite", "ellipse", "ellipse-hard") else "fp64"
    spec["precision"] = precision
    spec["layout"] = "stored" if precision == "tensor" else "matrix_free"
    # residual target: 1e-8 on ||f - A x|| / ||f|| keeps the error against the
    # FP64 solution below 1e-6 for the condition numbers of these operators
    spec["rtol"] = spec.get("rtol", 1e-8)
    spec["restart"] = 80
    spec["maxit"] = 4000
    return spec


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# roofline helpers
# ---------------------------------------------------------------------------
def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# Algorithmic work per (target, source) pair of each kernel class, counted from
# the kernels' per-pair formulas (FP32 add / mul / fma / min / max / rint and
# each special-function unit op = 1 operation, IEEE division or square root = 8).
SMS, FP32_LANES = 152, 128
# FP32 pair entries (two-float phase, asymptotics) by summation variant: the
# CUDA-core kernel evaluates both hard entries from one phase; the tensor-core
# kernel folds the per-node factors in, keeps the accuracy of its bf16 hi + lo
# operands (two-term series, no exact sum in the phase) and evaluates S (36)
# and D' (42) in two passes
ENTRY_OPS = {("soft", 1): 74, ("hard", 1): 87, ("soft", 2): 54, ("hard", 2): 36 + 42}
SUM_OPS = {"soft": 4, "hard": 8}         # FP32 FMAs per pair and right-hand side (CUDA-core sums)
DF_ENTRY_OPS = 563                       # double-float pair entry of the residual kernel
# sound hard: the phase and Hankel part (431) with the S assembly (39) and the D'
# assembly (78); the CUDA-core kernel takes both from one phase, the sliced
# tensor-core kernel evaluates them in separate passes
DF_HARD_OPS = 431 + 39 + 78
DF_HARD_PASS_OPS = (431 + 39) + (431 + 78)
DF_TERM_OPS = 48                         # Dot2 complex product-sum per pair and right-hand side
SLICE_OPS = 48                           # six 8-bit slices of the re / im parts of one entry
FP64_NOMINAL_TFLOPS = 1.25               # GB300 FP64 (nominal; FMA = 2 flops)


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from one
# ncu capture of the current kernel at the same launch configuration, keyed by
# (kernel class, curve, n, nrhs, matvec variant); absent = not captured.
NCU_TRAFFIC = {
    ("matvec_fp32", "kite", 32768, 64, 2): 79.033088e6 + 11.152128e6,
    ("matvec_fp64", "kite", 32768, 64, 2): 3.288266e9 + 157.754112e6,
}


def kernel_rooflines(kt, spec, stats, peaks, src, n, solves_timed):
    """Roofline entry per timed kernel class: achieved = algorithmic work of the
    class in the timed region / its CUDA-event time."""
    nrhs, bc, prec = spec["nrhs"], spec["bc"], spec["precision"]
    clock_hz = peaks.get("sm_max_mhz", 2070.0) * 1e6
    fp32_peak = SMS * FP32_LANES * clock_hz / 1e12        # T lane-ops/s
    out = {}
    variant = stats.get("matvec_variant", 0)
    for cls, (ms, launches) in kt.items():
        if launches == 0 or ms <= 0:
            continue
        sec = ms / 1e3
        avg = sec / launches
        if cls == "matvec_fp32":
            v = stats.get("matvec_variant", 1)
            ops = ENTRY_OPS[(bc, 2 if v == 2 else 1)] + (SUM_OPS[bc] * nrhs if v == 1 else 0)
            # per matvec (the sound-hard tensor-core form, and passes of more
            # than 64 right-hand sides, take several launches per matvec)
            mv = stats.get("inner_matvecs", 0) * solves_timed
            a = ops * n * n / (sec / mv if mv else avg) / 1e12
            out[cls] = {"bound": "alu", "achieved": a, "peak": fp32_peak, "unit": "Top/s",
                        "frac": a / fp32_peak, "traffic": None,
                        "work": f"{ops} FP32 ops per pair (variant {v}: "
                                + ("source sums on the tensor cores, not counted" if v == 2
                                   else f"{SUM_OPS[bc]} FMA per pair per right-hand side") + ")",
                        "peak_source": f"152 SMs x 128 FP32 lanes x {clock_hz / 1e6:.0f} MHz"}
        elif cls == "matvec_fp64" and prec != "fp64" and stats.get("residual_variant") == 2:
            ent, sl = (DF_ENTRY_OPS, SLICE_OPS) if bc == "soft" else (DF_HARD_PASS_OPS, 2 * SLICE_OPS)
            ops = ent + sl
            a = ops * n * n / avg / 1e12
            out[cls] = {"bound": "alu", "achieved": a, "peak": fp32_peak, "unit": "Top/s",
                        "frac": a / fp32_peak, "traffic": None,
                        "work": f"tensor-core residual: {ent} + {sl} FP32 ops per pair "
                                "(double-float entries, slicing; slice products on the tensor "
                                "cores, not counted)",
                        "peak_source": f"152 SMs x 128 FP32 lanes x {clock_hz / 1e6:.0f} MHz"}
        elif cls == "matvec_fp64" and prec != "fp64":
            # S applied to the 3 vectors of Maue's identity and D' to x: 4 sums per RHS
            ent, terms = (DF_ENTRY_OPS, 1) if bc == "soft" else (DF_HARD_OPS, 4)
            ops = ent + DF_TERM_OPS * terms * nrhs
            a = ops * n * n / avg / 1e12
            out[cls] = {"bound": "alu", "achieved": a, "peak": fp32_peak, "unit": "Top/s",
                        "frac": a / fp32_peak, "traffic": None,
                        "work": f"double-float residual: {ent} + {DF_TERM_OPS * terms} x nrhs "
                                "FP32 ops per pair",
                        "peak_source": f"152 SMs x 128 FP32 lanes x {clock_hz / 1e6:.0f} MHz"}
        elif cls == "matvec_fp64":
            dfma = (4 if bc == "soft" else 8) * nrhs
            a = dfma * n * n / avg / 1e12
            pk = FP64_NOMINAL_TFLOPS / 2
            out[cls] = {"bound": "alu", "achieved": a, "peak": pk, "unit": "T DFMA/s",
                        "frac": a / pk, "traffic": None,
                        "work": f"{dfma} DFMA per pair (source sums only: a lower bound)",
                        "peak_source": "nominal GB300 FP64 1.25 TFLOP/s (not measured)"}
        elif cls == "matvec_tensor":
            pitch = (n + 63) // 64 * 64
            b = n * pitch * 8
            a = b / avg / 1e9
            out[cls] = {"bound": "hbm", "achieved": a, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                        "frac": a / peaks["hbm_gbs"], "traffic": None,
                        "work": "stored bf16 hi/lo matrix (8 bytes per entry) read once per matvec",
                        "peak_source": src}
        elif cls == "arnoldi":
            elems = stats.get("arnoldi_elems", 0) * solves_timed
            esize = 8 if stats.get("basis_fp32") else 16
            b = 4 * elems * esize
            a = b / sec / 1e9
            e = {"bound": "hbm", "achieved": a, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                 "frac": a / peaks["hbm_gbs"], "traffic": None,
                 "work": f"CGS2: 4 passes over the basis, {esize} bytes per element",
                 "peak_source": src}
            if esize == 16:
                f = 20 * elems / sec / 1e12
                e["fp64_ops"] = {"achieved": f, "peak": FP64_NOMINAL_TFLOPS / 2,
                                 "unit": "T FP64 ops/s", "frac": f / (FP64_NOMINAL_TFLOPS / 2)}
            out[cls] = e
    for cls, e in out.items():
        e["traffic"] = NCU_TRAFFIC.get((cls, spec["curve"], n, nrhs, variant))
    return out


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def run_ours(args, rank, world):
    import numpy as np
    import torch

    from paper_1408_1578_gb300 import cfie, inputs

    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    spec = workload(args.workload, args.precision, args.n, args.nrhs, args.eta_factor)
    if args.rtol:
        spec["rtol"] = args.rtol
    if args.block:
        spec["restart"] = 40       # block steps per cycle
        spec["solver"] = "block GMRES"
    if args.fp64_basis:
        spec["solver"] = (spec.get("solver", "") + ", " if spec.get("solver") else "") + \
            "FP64 inner basis"
    n, w, nrhs, bc = spec["n"], spec["omega"], spec["nrhs"], spec["bc"]
    stream = torch.cuda.current_stream()
    ctx = cfie.Context(dev, stream=stream)
    prec_q = None
    if args.dirprec:
        # Section 2's node set: n = 4^q p points equispaced in arclength, p = 8
        prec_q = dirprec_levels(n, DIRPREC_P)
        if bc != "soft" or prec_q is None:
            raise SystemExit("--dirprec needs a sound-soft workload with n = 4^q * 8")
        arc = cfie.arclength_samples(spec["curve"], n, **spec["params"])
        spec["nodes"] = "arclength"
    else:
        arc = None
    setup_s = []
    theta = inputs.directions(nrhs)
    f = torch.empty((nrhs, n), dtype=torch.complex128, device="cuda")
    x = torch.zeros((nrhs, n), dtype=torch.complex128, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    # inputs larger than L2?  the Krylov basis is (restart+1) n nrhs 16 bytes
    basis_bytes = (spec["restart"] + 1) * n * nrhs * 16
    flush_l2 = basis_bytes < 2 * 129 * 1024 * 1024

    def step(precondition=True):
        if arc is None:
            geom = ctx.geometry(spec["curve"], **spec["params"])
        else:
            geom = ctx.samples(*arc[:3])
        op = geom.discretise(n, w, eta=spec["eta"], bc=bc, precision=spec["precision"],
                             layout=spec["layout"])
        if args.block:
            op.set_block_gmres(True)
        if args.fp64_basis:
            op.set_inner_basis(False)
        prec = None
        if arc is not None and precondition:
            t0 = time.perf_counter()
            prec = op.dirprec(spec["curve"], prec_q, DIRPREC_P, **spec["params"])   # synchronous
            setup_s.append(time.perf_counter() - t0)
            op.set_preconditioner(prec)
        op.rhs_plane_waves(theta, f)
        x.zero_()
        its, rel, st = op.gmres_solve(f, x, rtol=spec["rtol"], restart=spec["restart"],
                                      maxit=spec["maxit"], allow_noconv=True)
        stats = op.last_stats()
        if prec is not None:
            op.set_preconditioner(None)
            prec.close()
        op.close()
        geom.close()
        return its, rel, stats

    pipes = ctx.measure_peaks()
    unprec = None
    if arc is not None:
        # the same solve without the preconditioner, once, for the iteration
        # counts n_n beside n_p (Tables 1 and 3)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        its0, rel0, stats0 = step(precondition=False)
        torch.cuda.synchronize()
        unprec = {"iterations": [int(v) for v in its0[:4]], "max_relres": float(np.max(rel0)),
                  "s_per_step": time.perf_counter() - t0, "solve_stats": stats0}
    for _ in range(args.warmup):
        its, rel, stats = step()
    barrier(world)
    torch.cuda.synchronize()
    clocks = ClockSampler(dev)
    clocks.start()
    ctx.set_profiling(True)
    launches0 = ctx.lib.cfie_launch_count()
    ms_total = 0.0
    pairs = 0
    solves = 0
    worst = 0.0
    for _ in range(args.steps):
        if flush_l2:
            flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        its, rel, stats = step()
        e1.record(stream)
        torch.cuda.synchronize()
        ms_total += e0.elapsed_time(e1)
        pairs += n * n * (stats["inner_matvecs"] + stats["fp64_matvecs"])
        solves += int(np.sum(rel <= spec["rtol"]))
        worst = max(worst, float(np.max(rel)))
    barrier(world)
    torch.cuda.synchronize()
    launches = ctx.lib.cfie_launch_count() - launches0
    ktimes = ctx.kernel_times()
    ctx.set_profiling(False)
    clk = clocks.stop()
    ms_max = allreduce_max(ms_total, world)
    pairs_all = allreduce_sum(pairs, world)

    # end to end through the C ABI with host buffers: host angles in, host
    # solution out (pinned), copies inside the timed region
    x_host = torch.empty((nrhs, n), dtype=torch.complex128, pin_memory=True)
    e2e_ms = 0.0
    e2e_pairs = 0
    for _ in range(args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        its_e, rel_e, stats_e = step()   # angles go host -> device inside the C call
        x_host.copy_(x, non_blocking=True)
        torch.cuda.synchronize()
        e2e_ms += (time.perf_counter() - t0) * 1e3
        e2e_pairs += n * n * (stats_e["inner_matvecs"] + stats_e["fp64_matvecs"])
    e2e_ms_max = allreduce_max(e2e_ms, world)
    e2e_pairs_all = allreduce_sum(e2e_pairs, world)

    result = None
    if rank == 0:
        dom = max(ktimes, key=lambda k: ktimes[k][0])
        peaks, src = measured_peaks()
        roofs = kernel_rooflines(ktimes, spec, stats, peaks, src, n, args.steps)
        if dom not in roofs and roofs:
            # the largest class with a counted work model (e.g. when the
            # spectral derivative of a small sound-hard case takes the most)
            dom = max(roofs, key=lambda k: ktimes[k][0])
        roof = dict(roofs.get(dom, {}), kernel=dom) if dom in roofs else None
        value = pairs_all / (ms_max / 1e3)
        result = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp32": "f32+f64", "fp64": "f64", "tensor": "bf16x3+f64"}[spec["precision"]],
            "data": "synthetic",
            "config": dict(single_config(spec, world),
                           l2="flushed between steps" if flush_l2 else "Krylov basis larger than L2"),
            "solves_per_s": solves * world / (ms_max / 1e3),
            "max_relres": worst,
            "iterations": [int(v) for v in its[:4]],
            "solve_stats": stats,
            "e2e": {"value": e2e_pairs_all / (e2e_ms_max / 1e3), "unit": UNIT,
                    "h2d_bytes_per_step": int(8 * (nrhs + sum(len(v) for v in
                                                              spec["params"].values()
                                                              if isinstance(v, list)))),
                    "d2h_bytes_per_step": int(nrhs * n * 16)},
            "gpu_launches": int(launches),
            "kernel_ms": {k: round(v[0], 3) for k, v in ktimes.items()},
            "kernel_launches": {k: v[1] for k, v in ktimes.items()},
            "roofline": roof,
            "kernel_rooflines": roofs,
            "pipe_rates_measured": {"sms": pipes["sms"],
                                    "fp32_fma_T_per_s": pipes["fp32_fma_per_s"] / 1e12,
                                    "mufu_T_per_s": pipes["mufu_per_s"] / 1e12,
                                    "fp64_fma_T_per_s": pipes["fp64_fma_per_s"] / 1e12},
            "clocks": clk,
        }
        if unprec is not None:
            result["dirprec"] = {"q": prec_q, "p": DIRPREC_P, "nodes": "arclength",
                                 "iterations_preconditioned": [int(v) for v in its[:4]],
                                 "setup_s_median": statistics.median(setup_s) if setup_s else None,
                                 "setup_s_first": setup_s[0] if setup_s else None,
                                 "unpreconditioned": unprec}
    ctx.close()
    return result


# ---------------------------------------------------------------------------
# reference arm: the FP64 oracle on the host cores, bounded sample
# ---------------------------------------------------------------------------
def oracle_sample(spec, rows_count):
    """Pair evaluations of the oracle on `rows_count` rows of the workload's
    operator (the oracle's per-row assembly and product with the right-hand
    sides); returns pair evaluations done and seconds."""
    import numpy as np

    from oracle import geometry, kress, operators
    from paper_1408_1578_gb300 import inputs

    n, w, bc = spec["n"], spec["omega"], spec["bc"]
    c = geometry.make(spec["curve"], n, **spec["params"])
    R = kress.kress_weights(n)
    X = inputs.random_density(n, spec["nrhs"], seed=5)
    rows = np.arange(rows_count) * (n // rows_count)
    t0 = time.perf_counter()
    if bc == "soft":
        A = operators.soft_rows(c, w, spec["eta"], rows, R)
        _ = A @ X.T
        pairs = rows_count * n
    else:
        S = operators.layer_rows(c, w, rows, "S", R)
        Dp = operators.layer_rows(c, w, rows, "Dp", R)
        _ = S @ X.T, Dp @ X.T
        pairs = rows_count * n
    return pairs, time.perf_counter() - t0


ORACLE_THREAD_ENV = {k: "1" for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS",
                                        "BLIS_NUM_THREADS", "NUMEXPR_NUM_THREADS")}


def _oracle_runs(args, budget_s, procs):
    """Run `procs` copies of the bounded oracle sample at once, each in a fresh
    interpreter with its BLAS pinned to one thread; returns their JSON results."""
    env = dict(os.environ, **ORACLE_THREAD_ENV)
    cmd = [sys.executable, os.path.abspath(__file__), "--oracle-budget", str(budget_s),
           "--workload", args.workload]
    for k in ("precision", "n", "nrhs", "count", "eta_factor"):
        v = getattr(args, k)
        if v is not None:
            cmd += [f"--{k.replace('_', '-')}", str(v)]
    running = [subprocess.Popen(cmd, env=env, stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                                text=True) for _ in range(procs)]
    out = []
    for pr in running:
        so, se = pr.communicate(timeout=900)
        if pr.returncode != 0:
            raise RuntimeError("oracle sample failed: " + se[-500:])
        out.append(json.loads(so.strip().splitlines()[-1]))
    return out


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_all_cores(args, budget_s):
    """The oracle on every host core at once: one bounded-sample process per
    core (one thread each), their rates added."""
    cores = host_cores()
    runs = _oracle_runs(args, budget_s, cores)
    return {"value": sum(q["value"] for q in runs), "unit": runs[0]["unit"], "cores": cores,
            "sample": f"{cores} processes at once, one thread each, each: " + runs[0]["sample"]}


def oracle_single_core(args, budget_s):
    """Time the oracle on one host core (BLAS pinned to one thread) on a
    bounded sample of the workload, then on every host core at once; returns
    the cpu_baseline object: the one-core figure, the all-core one beside it."""
    r = _oracle_runs(args, budget_s, 1)[0]
    return {"value": r["value"], "unit": r["unit"], "cores": 1, "kind": "oracle",
            "sample": r["sample"], "all_cores": oracle_all_cores(args, budget_s)}


def oracle_budget_main(args):
    if args.workload == "serve":
        from oracle import geometry, operators, solvers
        from paper_1408_1578_gb300 import inputs
        reqs = inputs.poisson_requests(count=args.count or 32, rate=200.0, seed=1578, n_lo=1024,
                                       n_hi=65536)
        solves, secs, done = 0, 0.0, []
        for r in sorted(reqs, key=lambda q: q["n"]):
            t0 = time.perf_counter()
            c = geometry.fourier_star(r["n"], r["a"], r["b"])
            A = operators.cfie_matrix(c, r["omega"], r["omega"], r["bc"])
            F = operators.plane_wave_rhs(c, r["omega"], inputs.directions(r["nrhs"]), r["bc"])
            solvers.lu_solve(A, F)
            secs += time.perf_counter() - t0
            solves += r["nrhs"]
            done.append(f"n={r['n']} {r['bc']} nrhs={r['nrhs']}")
            if secs > args.oracle_budget:
                break
        print(json.dumps({"value": solves / secs, "unit": "solves/s",
                          "sample": f"dense LU solves of the smallest requests ({secs:.1f} s, one "
                                    "thread): " + "; ".join(done)}), flush=True)
        return
    specs = reference_specs(args)
    pairs, secs, parts = 0, 0.0, []
    for sp in specs:
        rows = cpu_rows_for(sp, budget_s=args.oracle_budget / len(specs))
        p, t = oracle_sample(sp, rows)
        pairs += p
        secs += t
        parts.append(f"{rows} rows x {sp['n']} sources of the {sp['name']} operator")
    print(json.dumps({"value": pairs / secs, "unit": UNIT,
                      "sample": "; ".join(parts) + f", {specs[0]['nrhs']} right-hand sides "
                                f"({secs:.1f} s, one thread)"}), flush=True)


def cpu_rows_for(spec, budget_s=12.0):
    pairs, secs = oracle_sample(spec, 4)
    rate = pairs / max(secs, 1e-6)
    rows = int(max(4, min(spec["n"], budget_s * rate / spec["n"])))
    return rows


def reference_specs(args):
    """Workloads the oracle samples: the named single-operator workload, or for
    the batch four of its stars (the smallest, the median and the two largest)."""
    if args.workload == "stars":
        from paper_1408_1578_gb300 import inputs
        stars = inputs.random_stars(count=args.count or 256, seed=1408, n_lo=512, n_hi=16384,
                                    nrhs=32)
        order = sorted(range(len(stars)), key=lambda k: stars[k]["n"])
        pick = [order[0], order[len(order) // 2], order[-2], order[-1]]
        return [{"name": f"stars[{k}]", "curve": "star",
                 "params": {"a": list(stars[k]["a"]), "b": list(stars[k]["b"])},
                 "n": stars[k]["n"], "omega": stars[k]["omega"], "nrhs": stars[k]["nrhs"],
                 "eta": stars[k]["omega"], "eta_factor": 1.0,
                 "bc": "soft", "precision": "tensor"} for k in pick]
    return [workload(args.workload, args.precision, args.n, args.nrhs, args.eta_factor)]


def run_reference_serve(args):
    """Served workload on the host: the oracle's dense LU solve of the smallest
    requests of the stream (assembly + LU + back substitution), solves/s."""
    import numpy as np

    from oracle import geometry, operators, solvers
    from paper_1408_1578_gb300 import inputs
    count = args.count or 32
    reqs = inputs.poisson_requests(count=count, rate=200.0, seed=1578, n_lo=1024, n_hi=65536)
    order = [int(i) for i in np.argsort([r["n"] for r in reqs])]
    solves, secs, done = 0, 0.0, []
    for step in range(args.warmup + args.steps):
        r = reqs[order[step % len(order)]]
        t0 = time.perf_counter()
        c = geometry.fourier_star(r["n"], r["a"], r["b"])
        A = operators.cfie_matrix(c, r["omega"], r["omega"], r["bc"])
        F = operators.plane_wave_rhs(c, r["omega"], inputs.directions(r["nrhs"]), r["bc"])
        solvers.lu_solve(A, F)
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            solves += r["nrhs"]
            secs += dt
            done.append(f"n={r['n']} {r['bc']} nrhs={r['nrhs']}")
    value = solves / secs
    return {
        "impl": "reference", "metric": SERVE_METRIC, "value": value, "unit": "solves/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": secs * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": serve_config(count),
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": 1, "kind": "oracle",
                         "sample": "dense LU solves of the smallest requests: " + "; ".join(done),
                         "all_cores": oracle_all_cores(args, 5.0)},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }


def run_reference(args, rank, world):
    if rank != 0:
        return None
    if args.workload == "serve":
        return run_reference_serve(args)
    specs = reference_specs(args)
    budget = 10.0 / max(1, args.steps + args.warmup) * 3 / len(specs)
    rows = [cpu_rows_for(sp, budget_s=budget) for sp in specs]
    for _ in range(args.warmup):
        for sp, r in zip(specs, rows):
            oracle_sample(sp, max(4, r // 4))
    tot_pairs, tot_s = 0, 0.0
    for _ in range(args.steps):
        for sp, r in zip(specs, rows):
            p, s = oracle_sample(sp, r)
            tot_pairs += p
            tot_s += s
    value = tot_pairs / tot_s
    sample = "; ".join(f"{r} rows x {sp['n']} sources of the {sp['name']} operator"
                       for sp, r in zip(specs, rows))
    sample += f", {specs[0]['nrhs']} right-hand sides, per step"
    cfg = stars_config(args.count or 256) if args.workload == "stars" else \
        single_config(workload(args.workload, args.precision, args.n, args.nrhs, args.eta_factor), world)
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot_s * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": cfg,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": sample, "all_cores": oracle_all_cores(args, 5.0)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


DIRPREC_P = 8   # points per wavelength of the paper's experiments (Section 3)


def dirprec_levels(n, p):
    """q with n = 4^q p, or None."""
    q, m = 0, n
    if m % p:
        return None
    m //= p
    while m > 1 and m % 4 == 0:
        m //= 4
        q += 1
    return q if m == 1 and q >= 1 else None


def single_config(spec, world):
    prec = " arclength nodes, directional preconditioner" if spec.get("nodes") == "arclength" else ""
    if spec.get("solver"):
        prec += ", " + spec["solver"]
    return {"workload": f"{spec['name']}: {spec['curve']} {spec['bc']} n={spec['n']} "
                        f"omega={spec['omega']} {eta_text(spec)} nrhs={spec['nrhs']}{prec}",
            "curve": spec["curve"], "bc": spec["bc"], "n": spec["n"], "omega": spec["omega"],
            "nrhs": spec["nrhs"], "eta": spec["eta"], "precision": spec["precision"],
            "rtol": spec["rtol"],
            "restart": spec["restart"], "parallelism": f"replicas{world}"}


def eta_text(spec):
    f = spec["eta_factor"]
    return "eta=omega" if f == 1.0 else f"eta={f:g}*omega"


def stars_config(count):
    return {"workload": f"stars: {count} random stars, n log-uniform [512, 16384], "
                        "10 ppw, 32 directions, stored tensor-core, lockstep GMRES",
            "rtol": 1e-8, "restart": 80, "parallelism": "replicas1"}


def serve_config(count):
    return {"workload": f"serve: {count} Poisson requests at 200/s, soft/hard, random "
                        "stars, n log-uniform [1024, 65536], 1..64 directions",
            "rtol": 1e-8, "restart": 80, "parallelism": "replicas1"}


# ---------------------------------------------------------------------------
# distributed plumbing (replicas only: barrier + max/sum of scalars)
# ---------------------------------------------------------------------------
_PG = None


def init_dist(backend=None):
    """Replicas: one process per GPU, no collective on the data path; the
    process group only carries the barrier and the max / sum of the timings."""
    global _PG
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        if backend is None:
            backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend)
        _PG = dist
    return rank, world


def _device():
    import torch
    return "cuda" if _PG is not None and _PG.get_backend() == "nccl" else "cpu"


def barrier(world):
    if world > 1:
        import torch
        if _device() == "cuda":
            _PG.barrier(device_ids=[torch.cuda.current_device()])
        else:
            _PG.barrier()


def _reduce(v, op, world):
    if world == 1:
        return v
    import torch
    t = torch.tensor([float(v)], device=_device(), dtype=torch.float64)
    _PG.all_reduce(t, op=op)
    return float(t.item())


def allreduce_max(v, world):
    return _reduce(v, _PG.ReduceOp.MAX if _PG else None, world)


def allreduce_sum(v, world):
    return _reduce(v, _PG.ReduceOp.SUM if _PG else None, world)


def main():
    args = parse()
    if args.eta_factor is not None and (args.eta_factor <= 0 or args.workload in ("stars", "serve")):
        sys.exit("--eta-factor takes a positive factor and applies to the single-operator workloads")
    if args.oracle_budget is not None:
        oracle_budget_main(args)
        return
    if args.impl == "reference":
        # the oracle runs on one host core: pin BLAS before numpy loads
        os.environ.update(ORACLE_THREAD_ENV)
    if args.workload in ("stars", "serve") and args.impl == "ours":
        out = run_stars(args) if args.workload == "stars" else run_serve(args)
        out["cpu_baseline"] = oracle_single_core(args, 12.0)
        print(json.dumps(out), flush=True)
        return
    rank, world = init_dist()
    if args.impl == "reference":
        out = run_reference(args, rank, world)
    else:
        out = run_ours(args, rank, world)
        if rank == 0 and out is not None and world == 1:
            out["cpu_baseline"] = oracle_single_core(args, 12.0)
            if default_headline(args):
                out["other_configs"] = run_other_configs(args)
    if rank == 0 and out is not None:
        print(json.dumps(out), flush=True)
    if _PG is not None:
        _PG.destroy_process_group()



def default_headline(args):
    """The plain headline run (the kite workload, no overrides), after which
    the other configurations are measured briefly."""
    return (args.workload == "kite" and not args.no_extras and args.precision is None
            and args.n is None and args.nrhs is None and args.eta_factor is None
            and args.rtol is None and not (args.block or args.dirprec or args.fp64_basis))


def _brief(r):
    keys = ("metric", "value", "unit", "steps", "warmup", "ms_per_step", "solves_per_s",
            "max_relres", "dtype", "gpu_launches", "clocks", "makespan_s", "p50_latency_s",
            "p99_latency_s", "p50_service_s", "failed", "contraction_tuning")
    out = {k: r[k] for k in keys if k in r}
    out["workload"] = r["config"]["workload"]
    if r.get("roofline"):
        rf = r["roofline"]
        out["roofline"] = {k: rf[k] for k in ("bound", "kernel", "achieved", "peak", "unit", "frac")
                           if k in rf}
    if "one_at_a_time_summary" in r:
        out["one_at_a_time_summary"] = r["one_at_a_time_summary"]
    return out


def run_other_configs(args):
    """Short runs of the suite's other configurations on the same GPU after the
    headline: the unit circle (FP64, unrestarted GMRES), the sound-hard star in
    the plain FP64 form and in the FP32 refined form, the 256-star stored batch,
    and the first 100 requests of the served stream.  Each single-operator and
    batch run keeps the timing rules (three warm-up steps, CUDA events, L2 as
    the headline run); steps = min(steps, 3)."""
    import copy
    out = {}

    def sub(workload, **kw):
        a = copy.copy(args)
        a.workload, a.precision, a.count, a.no_extras = workload, None, None, True
        a.steps, a.warmup = min(args.steps, 3), max(3, min(args.warmup, 3))
        for k, v in kw.items():
            setattr(a, k, v)
        return a

    runs = [("disk_fp64", lambda: run_ours(sub("disk"), 0, 1)),
            ("star_hard_fp64", lambda: run_ours(sub("star"), 0, 1)),
            ("star_hard_fp32", lambda: run_ours(sub("star", precision="fp32"), 0, 1)),
            ("stars256_stored", lambda: run_stars(sub("stars"))),
            ("serve_first100", lambda: run_serve(sub("serve", count=100)))]
    for name, fn in runs:
        # a failure here is reported beside the headline, which stands
        try:
            out[name] = _brief(fn())
        except Exception as e:   # noqa: BLE001
            out[name] = {"error": f"{type(e).__name__}: {e}"[:300]}
    return out


# ---------------------------------------------------------------------------
# extra workloads: the batched stored path and the request server
# ---------------------------------------------------------------------------
def run_stars(args):
    """256 random stars, stored bf16 hi/lo matrices, 32 directions each, all
    solved in lockstep (one persistent tensor-core launch per block matvec)."""
    import numpy as np
    import torch

    from paper_1408_1578_gb300 import cfie, inputs
    count = args.count or 256
    specs = inputs.random_stars(count=count, seed=1408, n_lo=512, n_hi=16384, nrhs=32)
    stream = torch.cuda.current_stream()
    ctx = cfie.Context(0, stream=stream)
    pairs_mv = sum(s["n"] ** 2 for s in specs)
    L = sum(s["n"] * s["nrhs"] for s in specs)
    f = torch.empty(L, dtype=torch.complex128, device="cuda")
    x = torch.zeros_like(f)

    tuning = {}

    def step():
        geoms = [ctx.fourier_star(s["a"], s["b"]) for s in specs]
        ops = ctx.discretise_many(geoms, [s["n"] for s in specs], [s["omega"] for s in specs],
                                  precision="tensor", layout="stored")
        for g in geoms:
            g.close()
        b = cfie.Batch(ctx, ops, [s["nrhs"] for s in specs])
        d, ms = b.tuning()
        tuning["dealing"] = ["round-robin", "greedy", "stream-K"][d]
        if any(ms):
            tuning["candidates_ms"] = dict(zip(["round-robin", "greedy", "stream-K"], ms))
        for k, s in enumerate(specs):
            ops[k].rhs_plane_waves(inputs.directions(s["nrhs"]), b.block(f, k))
        x.zero_()
        its, rel, _ = b.gmres_solve(f, x, rtol=1e-8, restart=80, maxit=4000, allow_noconv=True)
        stats = b.last_stats()
        b.close()
        for op in ops:
            op.close()
        return its, rel, stats

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    ctx.set_profiling(True)
    l0 = ctx.lib.cfie_launch_count()
    ms, pairs, solves, worst = 0.0, 0, 0, 0.0
    for _ in range(args.steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        its, rel, stats = step()
        e1.record(stream)
        torch.cuda.synchronize()
        ms += e0.elapsed_time(e1)
        pairs += pairs_mv * (stats["inner_matvecs"] + stats["fp64_matvecs"])
        solves += int(np.sum(rel <= 1e-8))
        worst = max(worst, float(np.max(rel)))
    kt = ctx.kernel_times()
    launches = ctx.lib.cfie_launch_count() - l0
    clk = clocks.stop()
    ctx.set_profiling(False)
    # end to end: host angles in (inside the C calls), solutions out to pinned
    # host memory, copies inside the timed region
    x_host = torch.empty(L, dtype=torch.complex128, pin_memory=True)
    e2e_ms, e2e_pairs = 0.0, 0
    for _ in range(args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        its_e, rel_e, stats_e = step()
        x_host.copy_(x, non_blocking=True)
        torch.cuda.synchronize()
        e2e_ms += (time.perf_counter() - t0) * 1e3
        e2e_pairs += pairs_mv * (stats_e["inner_matvecs"] + stats_e["fp64_matvecs"])
    peaks, src = measured_peaks()
    tens_ms, tens_n = kt["matvec_tensor"]
    gemm_bytes = sum(s["n"] * ((s["n"] + 63) // 64 * 64) * 8 for s in specs)   # n x pitch x 8
    roof = None
    if tens_n:
        gbs = gemm_bytes / (tens_ms / tens_n / 1e3) / 1e9
        roof = {"bound": "hbm",
                "kernel": "stored contraction graph (B preparation + k_gemm_persistent "
                          "[+ reduction for stream-K])",
                "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": gbs / peaks["hbm_gbs"], "traffic": None, "peak_source": src,
                "bytes_per_launch": gemm_bytes}
    out = {"metric": METRIC, "value": pairs / (ms / 1e3), "unit": UNIT, "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "bf16x3+f64", "data": "synthetic",
           "config": dict(stars_config(count), sum_n2=pairs_mv),
           "solves_per_s": solves / (ms / 1e3), "max_relres": worst, "solve_stats": stats,
           "e2e": {"value": e2e_pairs / (e2e_ms / 1e3), "unit": UNIT,
                   "h2d_bytes_per_step": int(sum(s["nrhs"] for s in specs) * 8),
                   "d2h_bytes_per_step": int(L * 16)},
           "gpu_launches": int(launches), "kernel_ms": {k: round(v[0], 3) for k, v in kt.items()},
           "kernel_launches": {k: v[1] for k, v in kt.items()}, "roofline": roof, "clocks": clk,
           "contraction_tuning": tuning}
    ctx.close()
    return out


def run_serve(args):
    """Poisson stream (200 requests/s) of sound-soft / sound-hard solves on random
    stars, n log-uniform in [1024, 65536], 1..64 directions, served by the
    library's request server (slots taking batches of compatible requests);
    p50 / p99 latency, solves/s.  A stated sample of the stream (its first
    requests with n <= 2560, the FP64 form being about 20x slower) is also run
    one request at a time in the served mixed-precision form and in the plain
    FP64 form."""
    import numpy as np
    import torch

    from paper_1408_1578_gb300 import cfie, inputs
    count = args.count or 32
    reqs = inputs.poisson_requests(count=count, rate=200.0, seed=1578, n_lo=1024, n_hi=65536)
    free, total = torch.cuda.mem_get_info()
    budget = int(0.8 * free)
    srv = cfie.Server(0, hbm_budget_bytes=budget, slots=args.serve_slots, batch=args.serve_batch,
                      block_min_rhs=args.serve_block_min, block_min_n=args.serve_block_min_n)

    def form(r):
        return "tensor" if r["bc"] == "soft" and r["n"] <= args.serve_stored_max_n else "fp32"

    clocks = ClockSampler(0)
    clocks.start()
    l0 = cfie.load().cfie_launch_count()
    t0 = time.perf_counter()
    tickets = []
    for r in reqs:
        delay = t0 + r["arrival"] - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        tickets.append(srv.submit(r["a"], r["b"], r["n"], r["omega"], nrhs=r["nrhs"], bc=r["bc"],
                                  rtol=1e-8, restart=80, maxit=4000, precision=form(r)))
    ok = srv.wait_all(7200)
    makespan = time.perf_counter() - t0
    launches = cfie.load().cfie_launch_count() - l0
    clk = clocks.stop()
    res = [srv.poll(t) for t in tickets]
    lat = np.array([q["latency_s"] for q in res])
    svc = np.array([q["service_s"] for q in res])
    que = np.array([q["queued_s"] for q in res])
    good = [q["status"] == cfie.CFIE_OK for q in res]
    solves = sum(r["nrhs"] for r, g in zip(reqs, good) if g)
    relres = max(q["relres_max"] for q in res)
    stats = srv.stats()
    srv.close()
    # a stated sample of the same stream one request at a time on an otherwise
    # idle GPU, served (mixed precision) form against the plain FP64 form
    sample = [i for i, r in enumerate(reqs) if r["n"] <= 2560][:12]
    cmp = []
    one = cfie.Server(0, hbm_budget_bytes=budget, slots=1, block_min_rhs=args.serve_block_min,
                      block_min_n=args.serve_block_min_n)
    plain = cfie.Server(0, hbm_budget_bytes=budget, slots=1)
    for i in sample:
        r = reqs[i]
        row = {"index": i, "n": r["n"], "nrhs": r["nrhs"], "bc": r["bc"]}
        row["form"] = form(r)
        for key, prec, sv in (("served", form(r), one), ("fp64", "fp64", plain)):
            t = sv.submit(r["a"], r["b"], r["n"], r["omega"], nrhs=r["nrhs"], bc=r["bc"],
                          rtol=1e-8, restart=80, maxit=4000, precision=prec)
            sv.wait_all(3600)
            q = sv.poll(t)
            row[key + "_alone_s"] = q["service_s"]
            row[key + "_ok"] = q["status"] == cfie.CFIE_OK
            sv.release(t)
        row["speedup"] = row["fp64_alone_s"] / row["served_alone_s"]
        cmp.append(row)
    one.close()
    plain.close()
    sub_solves = sum(c["nrhs"] for c in cmp)
    in_stream = sum(res[c["index"]]["service_s"] for c in cmp)
    cmp_summary = {
        "sample": "the first %d requests of the stream with n <= 2560 (arrival order), "
                  "each alone on the GPU" % len(cmp),
        "requests": len(cmp), "solves": sub_solves,
        "served_form_alone_solves_per_s": sub_solves / sum(c["served_alone_s"] for c in cmp),
        "fp64_solves_per_s": sub_solves / sum(c["fp64_alone_s"] for c in cmp),
        "served_in_stream_service_s": in_stream,
        "all_ok": all(c["served_ok"] and c["fp64_ok"] for c in cmp)} if cmp else {}
    return {"metric": SERVE_METRIC,
            "value": solves / makespan, "unit": "solves/s", "n_gpus": 1, "steps": 1, "warmup": 0,
            "higher_is_better": True, "data": "synthetic", "dtype": "f32+f64",
            "config": dict(serve_config(count), slots=args.serve_slots, batch=args.serve_batch,
                           stored_max_n=args.serve_stored_max_n,
                           block_min_rhs=args.serve_block_min,
                           block_min_n=args.serve_block_min_n, budget_bytes=budget),
            "forms": {"tensor": sum(form(r) == "tensor" for r in reqs),
                      "fp32": sum(form(r) == "fp32" for r in reqs)},
            "all_done": bool(ok), "requests_per_s": count / makespan, "makespan_s": makespan,
            "arrival_span_s": reqs[-1]["arrival"],
            "p50_latency_s": float(np.percentile(lat, 50)),
            "p99_latency_s": float(np.percentile(lat, 99)),
            "p50_queued_s": float(np.percentile(que, 50)),
            "p50_service_s": float(np.percentile(svc, 50)),
            "p99_service_s": float(np.percentile(svc, 99)),
            "max_relres": relres, "failed": int(len(good) - sum(good)),
            "server": stats, "fp64_one_at_a_time": cmp, "one_at_a_time_summary": cmp_summary,
            "gpu_launches": int(launches),
            "clocks": clk}

if __name__ == "__main__":
    main()
